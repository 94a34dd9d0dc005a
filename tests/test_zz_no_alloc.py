"""ghb_gram_noalloc: the Gram energies for callers that cannot allocate device
memory (inside another framework's arena, with memory reserved to the last
byte, or under a no-allocation policy).  Its scratch is a fixed 32 MiB device
array; the result must equal the allocating entry point ghb_gram within the
Gram parity tolerance (1e-12 relative), on two calls in a row (the second call
finds the first call's leftovers in the shared scratch).

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("case", [
    dict(d=2, N=[45, 31], inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 100.0),
                                      (0, (-0.3, -0.3, 0), (0.2, 0.1, 1), 4.0)]),
    dict(d=3, N=[9, 7, 11], inclusions=[(2, (0.1, -0.2, 0.05), (0.25, 0, 0), 30.0)]),
])
@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_gram_matches_allocating_entry_point(ghb, case, kind):
    d = case["d"]
    ctx = ghb.Context(d, case["N"], 1.0, case["inclusions"])
    rng = np.random.default_rng(17 + d + kind)
    fields = [torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(W.random_field(rng, d, case["N"])))).cuda()
              for _ in range(d)]
    grid = ctx.grid_values(kind)
    ref = ctx.gram(kind, fields)                      # ghb_gram (allocating)
    for _ in range(2):                                # two calls in a row
        got = ghb.gram_noalloc(d, ctx.N, ctx.M, grid, fields)
        assert got.shape == ref.shape
        assert rel(got, ref) < 1e-12
    sub = ghb.gram_noalloc(d, ctx.N, ctx.M, grid, fields[:1])
    assert rel(sub, ref[:1, :1]) < 1e-12


def test_noalloc_rejects_sizes_beyond_scratch(ghb):
    import paper_1412_2033_gb300.ghb as gb
    lib = gb.load_library()
    N = (ctypes.c_int * 3)(1023, 1023, 1)          # two fields need 2 x 33.5 MB of intermediates
    M = (ctypes.c_int * 3)(2048, 2048, 1)
    dummy = (ctypes.c_void_p * 3)(16, 16, 16)          # never dereferenced: rejected first
    out = (ctypes.c_double * 9)()
    st = lib.ghb_gram_noalloc(2, N, M, ctypes.c_void_p(16), 2, dummy, out, None)
    assert st == gb.GHB_ERR_INVALID
    assert b"scratch" in lib.ghb_last_error()
