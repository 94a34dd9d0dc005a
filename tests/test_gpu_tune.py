"""The autotuner's choices and every launch configuration against the oracle.

Any configuration computes the same operator (only rounding differs), so the
FP64 operator matches the oracle to 1e-12 and the FP32 one to 2e-5 relative
under each forced choice of radix grouping, column tile, rows per CTA and
specialised or runtime-plan kernels."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import coefficients as OC
from oracle import galerkin as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    yield g
    g.tune_reset()


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("M", [162, 256, 500, 4374])
def test_autotuned_configuration_is_valid(ghb, M):
    cfg = ghb.tune_get(M)
    assert cfg["cap32"] in (18, 32) and cfg["cap64"] in (9, 18)
    assert cfg["tile32"] == 0 and cfg["tile64"] == 0   # chosen per operand at launch
    assert cfg["rows32"] in (1, 2)
    if M not in (162, 486, 1458, 4374):
        assert cfg["ct_col"] == 0 and cfg["ct_row"] == 0
    assert ghb.tune_get(M) == cfg                   # stored, not re-tuned


CASES = [(81, 162), (127, 256)]      # N, M: specialised and runtime-plan lengths


@pytest.mark.parametrize("N,M", CASES)
def test_every_configuration_matches_the_oracle(ghb, N, M):
    m = W.random_disk_instance(11 + N, N=N)
    x = W.random_field(np.random.default_rng(N + 1), 2, [N, N])
    ref = ghb.half_from_full(OG.Operator(OC.material_from_dict(m), [N, N], OG.PRIMAL, M=[M, M]).apply(x))
    ct_opts = [0, 1] if M in (162, 486, 1458, 4374) else [0]
    tiles = [0, 1, 2, 4, 8, 16]   # 0: by the operand's shape
    checked = 0
    try:
        for cap, tile, rows, ct in itertools.product([9, 18, 32], tiles, [1, 2], ct_opts):
            ghb.tune_set(M, cap32=cap, tile32=tile, rows32=rows, ct_col=ct, ct_row=ct, cap64=min(cap, 18),
                         tile64=min(tile, 8))
            ctx = ghb.Context.from_microstructure(m)
            assert ctx.M == [M, M]
            for dt, tol in [(torch.complex64, 2e-5), (torch.complex128, 1e-12)]:
                xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
                got = ctx.matvec(xt).cpu().numpy()
                assert rel(got, ref) < tol, (cap, tile, rows, ct, dt)
            ctx.close()
            checked += 1
    finally:
        ghb.tune_reset()
    assert checked >= 30
