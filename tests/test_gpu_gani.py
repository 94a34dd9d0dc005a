"""GPU parity of the GaNi scheme (Def. GaNi, Algorithm 1) and its a-posteriori
bounds (eq. GaNi_apost) against the oracle (oracle/gani.py).

Tolerances: the FP64 operator 1e-12 and the FP32 one 2e-5 relative to the
largest entry, as for the Ga operator; the FP64 bounds and GaNi matrices
1e-11 relative with both sides' CG at relative residual 1e-13 (the exact
energy of the GaNi minimiser moves to first order with it); mixed precision
1e-8 relative."""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients as OC
from oracle import gani as GN

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "square_N15": dict(d=2, N=[15, 15], a0=1.0, inclusions=[(0, (0, 0, 0), (2 ** -0.5, 2 ** -0.5, 1), 10.0)]),
    "disk_ragged": dict(d=2, N=[25, 15], a0=1.0, inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 100.0)]),
    "d3_sphere_box": dict(d=3, N=[7, 9, 5], a0=2.0, inclusions=[
        (2, (0.1, -0.2, 0.05), (0.25, 0, 0), 9.0), (0, (-0.3, 0.3, -0.3), (0.2, 0.3, 0.25), 0.2)]),
}


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", ["primal", "dual"])
@pytest.mark.parametrize("project", [True, False])
def test_gani_operator_parity(ghb, name, kind, project):
    m = CASES[name]
    N = m["N"]
    op = GN.GaNiOperator(OC.material_from_dict(m), N, kind)
    x = W.random_field(np.random.default_rng(len(name) + 3), m["d"], N)
    ref = ghb.half_from_full(op.apply(x, project_out=project))
    ctx = ghb.Context.from_microstructure(m)
    k = ghb.GHB_GANI_PRIMAL if kind == "primal" else ghb.GHB_GANI_DUAL
    for dt, tol in [(torch.complex128, 1e-12), (torch.complex64, 2e-5)]:
        xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
        got = ctx.matvec(xt, kind=k, project=project).cpu().numpy()
        assert rel(got, ref) < tol, (name, kind, project, dt)


def test_gani_operator_full_size_sampled(ghb):
    """N = 729 (M = N = 729 for GaNi): the GaNi operator at sampled output
    frequencies against the periodic convolution with the samples' DFT."""
    N = 729
    m = W.centred_disk(N, fraction=0.3, value=100.0)
    ctx = ghb.Context.from_microstructure(m)
    x = W.random_field(np.random.default_rng(5), 2, [N, N])
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).cuda()
    y = ctx.matvec(xt, kind=ghb.GHB_GANI_PRIMAL, project=False).cpu().numpy()
    a = GN.sample_values(OC.material_from_dict(m), [N, N])
    ahat = np.fft.fft2(a) / a.size                       # a~(m), m mod N (library FFT on the samples)
    c = (N - 1) // 2
    k = np.arange(-c, c + 1)
    for l in [(0, 0), (3, 1), (-c, c), (200, 17)]:
        idx = np.ix_((l[0] - k) % N, (l[1] - k) % N)
        ref = [np.sum(ahat[idx] * x[comp]) for comp in range(2)]
        got = y[:, l[0] + c, l[1]]
        assert np.abs(got - ref).max() < 1e-11 * np.abs(x).sum() * np.abs(ahat).max()


@pytest.mark.parametrize("name", list(CASES))
def test_gani_bounds_fp64(ghb, name):
    m = CASES[name]
    mat = OC.material_from_dict(m)
    up, lo, A, Binv, _ = GN.gani_bounds(mat, m["N"], tol=1e-13)
    ctx = ghb.Context.from_microstructure(m, tol=1e-13)
    gup, glo, gA, gB, infos, st = ctx.bounds_gani()
    assert st == 0
    for got, ref in [(gup, up), (glo, lo), (gA, A), (gB, Binv)]:
        assert rel(got, ref) < 1e-11, (name, got, ref)
    # GaNi duality (Remark duality_gani) and Ga inside the a-posteriori bounds, on the GPU values
    assert rel(gB, gA) < 1e-9
    U, L, _, _ = ctx.bounds()
    scale = np.abs(gA).max()
    for small, big in [(glo, L), (L, U), (U, gup)]:
        assert np.linalg.eigvalsh(big - small).min() > -1e-10 * scale


def test_gani_bounds_mixed(ghb):
    m = CASES["disk_ragged"]
    up, lo, A, Binv, _ = GN.gani_bounds(OC.material_from_dict(m), m["N"], tol=1e-13)
    ctx = ghb.Context.from_microstructure(m, precision="mixed")
    gup, glo, gA, gB, infos, st = ctx.bounds_gani()
    assert st == 0 and all(i["outer_iters"] >= 1 for i in infos)
    for got, ref in [(gup, up), (glo, lo), (gA, A), (gB, Binv)]:
        assert rel(got, ref) < 1e-8


def test_gani_needs_small_prime_factors(ghb):
    m = dict(d=2, N=[37, 15], a0=1.0, inclusions=[])
    ctx = ghb.Context.from_microstructure(m)
    with pytest.raises(ghb.GhbError):
        ctx.bounds_gani()
    U, L, _, _ = ctx.bounds()                      # the Ga path is unaffected
    assert np.allclose(U, np.eye(2)) and np.allclose(L, np.eye(2))
