"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
* FP64 coefficient tables, double-grid values and operator applications:
  1e-12 relative to the largest entry (FP64 rounding of transforms of length
  <= 4374 stays below 1e-13; 1e-12 leaves a margin of ten).
* FP32 operator: 2e-5 relative to the largest entry (float epsilon 6e-8 times
  about 20 radix stages and the conditioning of the multiply).
* FP64 bounds: 1e-12 relative (the stated FP64 parity target).
* Mixed bounds: 1e-8 relative, upper >= oracle (1 - s), lower <= oracle (1 + s)
  with s the one-sided slack of tests/conftest.py (1e-13).
"""
import zlib

import numpy as np
import pytest

from conftest import one_sided_margins, one_sided_slack

import workloads as W
from oracle import coefficients as OC
from oracle import galerkin as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


MICROS = {
    "d2_box_disk": dict(d=2, N=[21, 17], a0=1.3, inclusions=[
        (0, (0.21, -0.13, 0), (0.35, 0.22, 1), 7.0), (1, (-0.27, 0.24, 0), (0.14, 0, 0), 25.0)]),
    "d2_square_M29": dict(d=2, N=[15, 15], a0=1.0, inclusions=[(0, (0, 0, 0), (2 ** -0.5, 2 ** -0.5, 1), 10.0)],
                          M=[29, 29]),
    "d2_disk_ragged": dict(d=2, N=[45, 31], a0=1.0, inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 100.0)]),
    "d3_sphere_box": dict(d=3, N=[7, 9, 5], a0=2.0, inclusions=[
        (2, (0.1, -0.2, 0.05), (0.2, 0, 0), 30.0), (0, (-0.3, 0.25, -0.3), (0.15, 0.2, 0.25), 0.5)]),
    "d3_sphere_15": dict(d=3, N=[15, 15, 15], a0=1.0, inclusions=[(2, (0, 0, 0), (0.3627832, 0, 0), 1000.0)]),
}


def make_ctx(ghb, spec, **opts):
    if "M" in spec:
        opts = dict(opts, M=tuple(spec["M"]))
    return ghb.Context(spec["d"], spec["N"], spec["a0"], spec["inclusions"], **opts)


def oracle_material(spec):
    return OC.material_from_dict(spec)


@pytest.mark.parametrize("name", list(MICROS))
def test_coefficient_table_parity(ghb, name):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec)
    mat = oracle_material(spec)
    for kind, m in ((ghb.GHB_PRIMAL, mat), (ghb.GHB_DUAL, mat.inverse())):
        tab = OC.coeff_table(m, spec["N"])
        Nd = spec["N"][-1]
        ref = tab[..., Nd - 1:]                     # n_d = 0..N_d-1
        got = ctx.table(kind).cpu().numpy()
        assert got.shape == ref.shape
        assert rel(got, ref) < 2e-14


@pytest.mark.parametrize("N,c", [(729, (0.0, 0.0)), (301, (0.137, -0.291))])
def test_disk_table_large_arguments(ghb, N, c):
    """Disk coefficients at J1 arguments up to 2 pi r |k| ~ 2000: the device's
    J1 (Miller recurrence / Hankel expansion beyond x = 8) and phase against the
    oracle (scipy's J1).  Both evaluate J1 at the same FP64 argument, so they
    agree to about 1e-15 of the envelope r sqrt(2/(pi x)) / |k|."""
    m = dict(d=2, N=[N, N], a0=1.0, inclusions=[(1, (c[0], c[1], 0), (0.3090194, 0, 0), 100.0)])
    ctx = ghb.Context.from_microstructure(m)
    tab = OC.coeff_table(OC.material_from_dict(m), m["N"])[..., N - 1:]
    got = ctx.table(ghb.GHB_PRIMAL).cpu().numpy()
    k = OC.freq_grid([2 * N - 1, 2 * N - 1])[..., N - 1:, :].astype(float)
    rho = np.maximum(np.sqrt((k ** 2).sum(-1)), 1.0)
    env = 99.0 * 0.3090194 / rho * np.sqrt(2 / (np.pi * 2 * np.pi * 0.3090194 * rho))
    assert np.abs(got - tab).max() / env.max() < 1e-13
    assert (np.abs(got - tab) / env).max() < 2e-14


@pytest.mark.parametrize("name", list(MICROS))
def test_double_grid_values_parity(ghb, name):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec)
    mat = oracle_material(spec)
    for kind, m in ((ghb.GHB_PRIMAL, mat), (ghb.GHB_DUAL, mat.inverse())):
        tab = OC.coeff_table(m, spec["N"])
        ref = OG.double_grid_values(tab, ctx.M)
        got = ctx.grid_values(kind).cpu().numpy()
        # each value is a sum over Z_{2N-1} of table entries, each allowed an error
        # of 1e-12 max|a^| by the table test, plus transform rounding
        # (eps log2(M) sum|a^| < 1e-14 sum|a^|)
        bound = tab.size * 1e-12 * np.abs(tab).max() + 1e-14 * np.abs(tab).sum()
        assert np.abs(got - ref).max() < bound


@pytest.mark.parametrize("name", list(MICROS))
@pytest.mark.parametrize("kind", ["primal", "dual"])
@pytest.mark.parametrize("project", [True, False])
def test_matvec_fp64_parity(ghb, name, kind, project):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec)
    rng = np.random.default_rng(zlib.crc32(f"{name}/{kind}".encode()))
    x = W.random_field(rng, spec["d"], spec["N"])
    op = OG.Operator(oracle_material(spec), spec["N"], OG.PRIMAL if kind == "primal" else OG.DUAL, M=ctx.M)
    ref = op.apply(x, project_out=project)
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).cuda()
    k = ghb.GHB_PRIMAL if kind == "primal" else ghb.GHB_DUAL
    y = ctx.matvec(xt, kind=k, project=project)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    assert rel(got, ghb.half_from_full(ref)) < 1e-12


@pytest.mark.parametrize("name", ["d2_box_disk", "d2_disk_ragged", "d3_sphere_box"])
def test_matvec_fp32_parity(ghb, name):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec)
    rng = np.random.default_rng(5)
    x = W.random_field(rng, spec["d"], spec["N"])
    op = OG.Operator(oracle_material(spec), spec["N"], OG.PRIMAL, M=ctx.M)
    ref = ghb.half_from_full(op.apply(x))
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(torch.complex64).cuda()
    got = ctx.matvec(xt, kind=ghb.GHB_PRIMAL).cpu().numpy()
    assert rel(got, ref) < 2e-5


@pytest.mark.parametrize("name", ["d2_box_disk", "d2_square_M29", "d3_sphere_box"])
def test_gram_energy_parity(ghb, name):
    """Gram of arbitrary Hermitian fields, a(v_i, v_j) on the double grid vs the
    oracle's dense-definition energy (Lemma integ_eval_VM)."""
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec)
    rng = np.random.default_rng(11)
    d = spec["d"]
    fields = [W.random_field(rng, d, spec["N"]) for _ in range(d)]
    op = OG.Operator(oracle_material(spec), spec["N"], OG.PRIMAL, M=ctx.M)
    ref = np.array([[OG.inner(op.apply(fields[i], project_out=False), fields[j]) for j in range(d)]
                    for i in range(d)])
    ft = [torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(f))).cuda() for f in fields]
    got = ctx.gram(ghb.GHB_PRIMAL, ft)
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("name", ["d2_box_disk", "d2_square_M29", "d2_disk_ragged", "d3_sphere_box"])
def test_bounds_fp64_parity(ghb, name):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec, tol=1e-12)
    U, L, infos, st = ctx.bounds()
    assert st == 0
    Uo, Lo, _ = OG.bounds(oracle_material(spec), spec["N"], M=ctx.M, tol=1e-12)
    assert rel(U, Uo) < 1e-12
    assert rel(L, Lo) < 1e-12
    assert all(i["status"] == 0 for i in infos)


@pytest.mark.parametrize("name", ["d2_box_disk", "d2_disk_ragged", "d3_sphere_15"])
def test_bounds_mixed_parity_and_one_sided(ghb, name):
    spec = MICROS[name]
    ctx = make_ctx(ghb, spec, tol=1e-10, precision="mixed")
    U, L, infos, st = ctx.bounds()
    assert st == 0
    Uo, Lo, _ = OG.bounds(oracle_material(spec), spec["N"], M=ctx.M, tol=1e-12)
    assert rel(U, Uo) < 1e-8 and rel(L, Lo) < 1e-8
    d = spec["d"]
    su, sl = one_sided_slack(spec)
    mu, ml = one_sided_margins(U, L, Uo, Lo)
    assert mu >= -su and ml >= -sl, (mu, ml, su, sl)
    assert np.all(np.linalg.eigvalsh(U - Uo) > -su * np.abs(Uo).max())
    assert any(i["matvecs_fp32"] > 0 for i in infos)


@pytest.mark.parametrize("name", ["d2_disk_ragged", "d2_square_M29", "d3_sphere_box"])
def test_mixed_gram_on_zn_matches_double_grid(ghb, name):
    """The mixed path forms its Gram matrices on Z_N from the final FP64
    residual application (unprojected operator output of each iterate plus
    a^(k) E_i); the same fields (the solves are deterministic) through the
    double-grid Gram passes give the same matrices to FP64 rounding."""
    spec = MICROS[name]
    d = spec["d"]
    ctx = make_ctx(ghb, spec, tol=1e-10, precision="mixed")
    U, L, infos, st = ctx.bounds()
    assert st == 0
    G = {}
    for kind in (ghb.GHB_PRIMAL, ghb.GHB_DUAL):
        fields = []
        for i in range(d):
            f, info, _, s = ctx.solve_ex(np.eye(d)[i], kind=kind)
            assert s == 0
            assert abs(info["energy"] - infos[kind * d + i]["energy"]) < 1e-13 * abs(info["energy"])
            fields.append(f)
        X = np.asarray(ctx.gram(kind, fields))
        G[kind] = 0.5 * (X + X.T)
    assert rel(U, G[ghb.GHB_PRIMAL]) < 1e-13
    assert rel(L, np.linalg.inv(G[ghb.GHB_DUAL])) < 1e-12


def test_homogeneous_and_trivial_order(ghb):
    ctx = ghb.Context(2, [9, 9], 3.5, [])
    U, L, infos, st = ctx.bounds()
    assert np.allclose(U, 3.5 * np.eye(2), rtol=0, atol=1e-14) and np.allclose(L, 3.5 * np.eye(2), atol=1e-14)
    assert all(i["iters"] == 0 for i in infos)
    # N = 1: no fluctuation is admissible, the bounds are Voigt and Reuss exactly
    m = W.centred_disk(1, value=20.0)
    mat = OC.material_from_dict(m)
    ctx1 = ghb.Context.from_microstructure(m)
    U1, L1, _, st = ctx1.bounds()
    assert abs(U1[0, 0] - mat.mean()) < 1e-13 * mat.mean()
    assert abs(L1[0, 0] - mat.harmonic_mean()) < 1e-13 * mat.harmonic_mean()


@pytest.mark.parametrize("d", [2, 3])
def test_laminate_closed_form_gpu(ghb, d):
    m = W.laminate(9 if d == 2 else 5, d=d, h=0.37, value=8.0, a0=1.5, center=0.11)
    arith = 1.5 + 6.5 * 0.37
    harm = 1.0 / (1 / 1.5 + (1 / 8.0 - 1 / 1.5) * 0.37)
    for prec in ("fp64", "mixed"):
        ctx = ghb.Context.from_microstructure(m, precision=prec)
        U, L, _, st = ctx.bounds()
        for a in range(1, d):
            assert abs(U[a, a] - arith) < 1e-13 * arith
        assert abs(L[0, 0] - harm) < 1e-13 * harm


def test_repeatable_bitwise(ghb):
    spec = MICROS["d2_box_disk"]
    ctx = make_ctx(ghb, spec)
    a = ctx.bounds()
    b = ctx.bounds()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# transform lengths exercising every pass shape of the planner: 162 = 2.3^4,
# 486 = 2.3^5, 256 = 4^4, 216 = 4.2.3^3, 125 = 5^3, 150 = 2.3.5^2, 4374 = 2.3^7
SIZES = [(81, None), (243, None), (127, None), (101, None), (63, None), (75, None)]


@pytest.mark.parametrize("N,M", SIZES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_sizes(ghb, N, M, prec):
    m = W.random_disk_instance(7 + N, N=N)
    ctx = ghb.Context.from_microstructure(m)
    x = W.random_field(np.random.default_rng(N), 2, [N, N])
    op = OG.Operator(OC.material_from_dict(m), [N, N], OG.PRIMAL, M=ctx.M)
    ref = ghb.half_from_full(op.apply(x))
    dt = torch.complex128 if prec == "f64" else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
    got = ctx.matvec(xt).cpu().numpy()
    assert rel(got, ref) < (1e-12 if prec == "f64" else 2e-5)


@pytest.mark.parametrize("N", [729, 2187])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_full_size_sampled(ghb, N, prec):
    """The measured workload (d = 2 disk, N = 2187, M = 4374) and N = 729
    (M = 1458): the operator on a random field at sampled output frequencies
    against the oracle's definition y(l) = G(l) sum_k a^(l - k) x(k)."""
    m = W.centred_disk(N, fraction=0.3, value=100.0)
    ctx = ghb.Context.from_microstructure(m)
    assert ctx.M == [2 * N, 2 * N]
    x = W.random_field(np.random.default_rng(N), 2, [N, N])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
    y = ctx.matvec(xt).cpu().numpy()
    c = (N - 1) // 2
    idx = np.array([[0, 0], [1, 0], [0, 1], [-c, c], [c, 0], [37, c - 182], [-512 % c, 3], [c - 393, c]])
    ref = OG.matvec_sampled(x, OC.material_from_dict(m), OG.PRIMAL, idx)
    got = np.array([y[:, l[0] + c, l[1]] for l in idx])
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < (1e-11 if prec == "f64" else 2e-5) * scale


# (N, double grid): the 3-D orders of the sphere/cube family and their
# size-specialised transform lengths 72 = 3^2 4 2, 135 = 5 3^3, 162 = 3^4 2,
# 270 = 5 3^3 2
D3_SIZES = [(33, 72), (65, 135), (81, 162), (129, 270)]


@pytest.mark.parametrize("N,M", D3_SIZES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_3d_specialised_sampled(ghb, N, M, prec):
    """d = 3 at N = 33 ... 129 (M = 72 ... 270 on every axis): the
    size-specialised column passes on both non-contiguous axes and the
    last-axis pass with three interleaved lines per CTA (FP32: A_M read in the
    fused pass), at sampled output frequencies against the oracle's definition
    y(l) = G(l) sum_k a^(l - k) x(k), primal and dual."""
    m = W.centred_sphere(N, fraction=0.2, value=1000.0)
    m["inclusions"].append((0, (0.38, -0.35, 0.33), (0.15, 0.2, 0.12), 0.3))   # a box clear of the sphere
    mat = OC.material_from_dict(m)
    ctx = ghb.Context.from_microstructure(m)
    assert ctx.M == [M] * 3
    x = W.random_field(np.random.default_rng(3 * N), 3, [N, N, N])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
    c = (N - 1) // 2
    idx = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [-c, c, c], [c, -3, 0], [7, -c, 11], [-13, 12, c]])
    for kind, okind in ((ghb.GHB_PRIMAL, OG.PRIMAL), (ghb.GHB_DUAL, OG.DUAL)):
        y = ctx.matvec(xt, kind=kind).cpu().numpy()
        ref = OG.matvec_sampled(x, mat if okind == OG.PRIMAL else mat.inverse(), okind, idx)
        got = np.array([y[:, l[0] + c, l[1] + c, l[2]] for l in idx])
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() < (1e-11 if prec == "f64" else 2e-5) * scale, (prec, kind)


# ragged 3-D orders that put one size-specialised length (M = 270 or 135) on
# each axis in turn, the others on runtime plans: every entry against the
# oracle's double-grid operator
RAGGED_3D = [([129, 9, 7], [270, 18, 15]), ([7, 129, 9], [15, 270, 18]), ([9, 7, 129], [18, 15, 270]),
             ([65, 11, 9], [135, 24, 18])]


@pytest.mark.parametrize("N,M", RAGGED_3D)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_3d_ragged_specialised(ghb, N, M, prec):
    m = dict(d=3, N=N, a0=1.0, inclusions=[(2, (0.1, -0.05, 0.2), (0.27, 0, 0), 40.0),
                                            (0, (-0.3, 0.3, -0.3), (0.2, 0.15, 0.1), 0.5)])
    ctx = ghb.Context.from_microstructure(m)
    assert ctx.M == M
    mat = OC.material_from_dict(m)
    x = W.random_field(np.random.default_rng(sum(N)), 3, N)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
    for kind, okind in ((ghb.GHB_PRIMAL, OG.PRIMAL), (ghb.GHB_DUAL, OG.DUAL)):
        ref = ghb.half_from_full(OG.Operator(mat, N, okind, M=M).apply(x))
        got = ctx.matvec(xt, kind=kind).cpu().numpy()
        assert rel(got, ref) < (1e-12 if prec == "f64" else 2e-5), (prec, kind)
