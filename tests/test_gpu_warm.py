"""GPU: bound tracking along CG and the coarse-to-fine start (Section 7.4)
against the oracle.

Tolerances: energies along FP64 CG 1e-9 relative to the oracle's energies by
definition over the first 30 iterates (both CGs run the same FP64 recurrences;
their iterates drift apart by rounding only); prolongation bitwise (a copy);
the warm start's first energy 1e-12 relative to the coarse bound (exact
energies on both grids); final bounds of warm and cold starts 1e-10."""
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
    return g


SQUARE = dict(d=2, N=[15, 15], a0=1.0, inclusions=[(0, (0, 0, 0), (2 ** -0.5, 2 ** -0.5, 1), 10.0)])
BALL_BOX = dict(d=3, N=[9, 7, 11], a0=2.0, inclusions=[
    (2, (0.1, -0.2, 0.05), (0.3, 0, 0), 50.0), (0, (-0.3, 0.3, -0.3), (0.2, 0.3, 0.25), 0.1)])


@pytest.mark.parametrize("kind", ["primal", "dual"])
@pytest.mark.parametrize("m", [SQUARE, BALL_BOX], ids=["square_N15", "d3_ball_box"])
def test_history_fp64_matches_oracle(ghb, kind, m):
    mat = OC.material_from_dict(m)
    E = [1.0, 0.4, -0.7][:m["d"]]
    op = OG.Operator(mat, m["N"], kind)
    _, info = OG.cg(op, op.rhs(E), 1e-10, track_energy_E=E)
    ref = np.array(info["energies"])
    ctx = ghb.Context.from_microstructure(m, tol=1e-10)
    k = ghb.GHB_PRIMAL if kind == "primal" else ghb.GHB_DUAL
    field, inf, en, st = ctx.solve_ex(E, kind=k, energies=True)
    assert st == 0 and len(en) == inf["iters"] + 1
    n = min(30, len(en), len(ref))
    assert np.abs(en[:n] - ref[:n]).max() < 1e-9 * ref[0]
    assert np.all(np.diff(en) <= 1e-12 * en[0])                      # monotone (CG minimises)
    assert abs(en[-1] - inf["energy"]) < 1e-10 * inf["energy"]       # ends at the exact energy
    voigt = (mat.mean() if kind == "primal" else mat.inverse().mean()) * float(np.dot(E, E))
    assert abs(en[0] - voigt) < 1e-13 * voigt                        # the Voigt (Reuss) start


@pytest.mark.parametrize("Nc,Nf", [([9, 7], [21, 15]), ([5, 7, 3], [9, 11, 7]), ([3, 3, 3], [3, 5, 9])])
def test_prolong_is_a_copy(ghb, Nc, Nf):
    rng = np.random.default_rng(4 + len(Nc))
    xc = W.random_field(rng, len(Nc), Nc)
    ref = ghb.half_from_full(OG.prolong(xc, Nf))
    xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(xc))).cuda()
    got = ghb.prolong(xt, Nf).cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("d,N,Nc", [(2, 81, 27), (3, 27, 9)])
def test_warm_start(ghb, precision, d, N, Nc):
    m = W.centred_disk(N, fraction=0.3, value=100.0) if d == 2 else W.centred_sphere(N, fraction=0.2, value=1000.0)
    mc = dict(m, N=[Nc] * d)
    E = [1.0] + [0.0] * (d - 1)
    cc = ghb.Context.from_microstructure(mc, precision=precision)
    fc, ic, _, _ = cc.solve_ex(E)
    ec = fc.clone()
    zero = (Nc - 1) // 2
    for i in range(d):                               # the fluctuation of the coarse field
        ec[(i,) + (zero,) * (d - 1) + (0,)] -= E[i]
    x0 = ghb.prolong(ec, [N] * d)
    cf = ghb.Context.from_microstructure(m, precision=precision)
    fw, iw, ew, sw = cf.solve_ex(E, x0=x0, energies=True)
    fz, iz, ez, sz = cf.solve_ex(E, energies=True)
    assert sw == 0 and sz == 0
    assert abs(ew[0] - ic["energy"]) < 1e-12 * ic["energy"]          # starts at the coarse bound
    assert ew[0] < ez[0]                                            # below the Voigt start
    assert np.all(np.diff(ew) <= 1e-12 * ew[0])
    assert abs(iw["energy"] - iz["energy"]) < 1e-10 * iz["energy"]  # same bound at the end
