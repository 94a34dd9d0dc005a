"""The C-ABI library loads and exports every symbol include/ghb.h declares;
host-side argument validation answers with the documented error codes
(these calls return before any CUDA work, so they run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_2033_gb300 import build
    build.build()
    import paper_1412_2033_gb300 as g
    return g.load_library()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ghb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ghb_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    import paper_1412_2033_gb300.ghb as gb
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(gb.EXPORTS) == syms


def test_version_and_defaults(lib):
    import paper_1412_2033_gb300.ghb as gb
    assert lib.ghb_version().startswith(b"ghb")
    o = gb.GhbOptions()
    lib.ghb_default_options(ctypes.byref(o))
    assert o.tol == 1e-10 and o.precision == gb.GHB_FP64 and list(o.M) == [0, 0, 0]
    assert ctypes.sizeof(gb.GhbOptions) == 40 and ctypes.sizeof(gb.GhbSolveInfo) == 40
    assert ctypes.sizeof(gb.GhbPhase) == 64


def _create(lib, d, N, a0, incs, **opt):
    import paper_1412_2033_gb300.ghb as gb
    h = ctypes.c_void_p()
    Nc = (ctypes.c_int * 3)(*(list(N) + [1] * (3 - len(N))))
    ph, n = gb.make_phases(incs)
    o = gb.Options(**opt).to_c()
    st = lib.ghb_create(ctypes.byref(h), d, Nc, a0, ph, n, ctypes.byref(o))
    return st, h, lib.ghb_last_error().decode()


@pytest.mark.parametrize("case", [
    dict(d=4, N=[5, 5], a0=1.0, incs=[]),
    dict(d=2, N=[4, 5], a0=1.0, incs=[]),                                      # even N
    dict(d=2, N=[5, 5], a0=-1.0, incs=[]),                                     # a0 <= 0
    dict(d=2, N=[5, 5], a0=1.0, incs=[(1, (0, 0, 0), (0.6, 0, 0), 2.0)]),      # r > 1/2
    dict(d=2, N=[5, 5], a0=1.0, incs=[(0, (0, 0, 0), (1.2, 0.5, 0), 2.0)]),    # box side > 1
    dict(d=2, N=[5, 5], a0=1.0, incs=[(2, (0, 0, 0), (0.2, 0, 0), 2.0)]),      # sphere in 2-D
    dict(d=2, N=[5, 5], a0=1.0, incs=[(1, (0.45, 0, 0), (0.1, 0, 0), 2.0),
                                       (1, (-0.45, 0, 0), (0.1, 0, 0), 2.0)]),  # periodic overlap
    dict(d=2, N=[5, 5], a0=1.0, incs=[(1, (0, 0, 0), (0.2, 0, 0), 0.0)]),      # zero coefficient
    dict(d=2, N=[5, 5], a0=1.0, incs=[], M=(8, 9, 0)),                         # M < 2N - 1
    dict(d=2, N=[5, 5], a0=1.0, incs=[], M=(37, 37, 0)),                       # prime factor > 31
    dict(d=2, N=[5, 5], a0=1.0, incs=[], tol=0.0),
])
def test_invalid_inputs_rejected(lib, case):
    opt = {}
    if "M" in case:
        opt["M"] = case["M"]
    if "tol" in case:
        opt["tol"] = case["tol"]
    st, h, msg = _create(lib, case["d"], case["N"], case["a0"], case["incs"], **opt)
    assert st == 1 and not h.value and msg


def test_null_arguments(lib):
    assert lib.ghb_create(None, 2, None, 1.0, None, 0, None) == 1
    assert lib.ghb_matvec(None, 0, 0, 1, None, None, None) == 1
    assert lib.ghb_bounds(None, None, None, None) == 1
    lib.ghb_destroy(None)


def test_tune_set_validation_and_size_rules(lib, monkeypatch):
    """Launch configurations: ghb_tune_set validates before storing, and with
    GHB_AUTOTUNE=0 ghb_tune_get answers with the size rules (no GPU work)."""
    import paper_1412_2033_gb300 as g
    monkeypatch.setenv("GHB_AUTOTUNE", "0")
    g.tune_reset()
    try:
        assert g.tune_get(4374) == dict(cap32=32, tile32=0, rows32=0, ct_col=1, ct_row=1, cap64=18, tile64=0)
        assert g.tune_get(510)["ct_col"] == 0                      # no specialised kernels at 510
        bad = [dict(cap32=4), dict(cap32=33), dict(tile32=3), dict(tile64=16), dict(rows32=3),
               dict(ct_col=2)]
        for b in bad:
            with pytest.raises(g.GhbError):
                g.tune_set(4374, **b)
        with pytest.raises(g.GhbError):
            g.tune_set(510, ct_row=1)                               # only for lengths that have them
        with pytest.raises(g.GhbError):
            g.tune_get(4373)                                        # prime > 31
        cfg = g.tune_set(510, cap32=18, tile32=4, rows32=1)
        assert g.tune_get(510) == cfg
    finally:
        g.tune_reset()


def test_gram_noalloc_binding_rejects_bad_arguments(lib):
    """The binding of ghb_gram_noalloc checks its arguments before the call:
    dimension, field count (1..d) and tensor kind (host tensors, wrong dtype,
    wrong size) are rejected with ValueError and never reach the library."""
    torch = pytest.importorskip("torch")
    import paper_1412_2033_gb300 as g
    grid = torch.zeros(100, dtype=torch.float64)
    f = torch.zeros(2 * 5 * 3, dtype=torch.complex128)
    with pytest.raises(ValueError):
        g.gram_noalloc(4, [5, 5], [10, 10], grid, [f])            # d not 2 or 3
    with pytest.raises(ValueError):
        g.gram_noalloc(2, [5, 5], [10, 10], grid, [])             # no field
    with pytest.raises(ValueError):
        g.gram_noalloc(2, [5, 5], [10, 10], grid, [f, f, f])      # more fields than d
    with pytest.raises(ValueError):
        g.gram_noalloc(2, [5, 5], [10, 10], grid, [f])            # host tensors
