"""GPU parity of the reduced form of the Ga operator (Lemma reduce_grid,
Algorithm 3): against the oracle, against the double-grid form on the GPU
(the same operator: equal up to rounding), and through the bounds.

Tolerances as for the double-grid operator: FP64 1e-12 and FP32 2e-5
relative to the largest entry; FP64 bounds 1e-12, mixed 1e-8."""
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


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


CASES = {
    "square_N15": (dict(d=2, N=[15, 15], a0=1.0, inclusions=[(0, (0, 0, 0), (2 ** -0.5, 2 ** -0.5, 1), 10.0)]), None),
    "disk_25x15": (dict(d=2, N=[25, 15], a0=1.0, inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 100.0)]), None),
    "d3_7x9x5": (dict(d=3, N=[7, 9, 5], a0=2.0, inclusions=[
        (2, (0.1, -0.2, 0.05), (0.25, 0, 0), 9.0), (0, (-0.3, 0.3, -0.3), (0.2, 0.3, 0.25), 0.2)]), [14, 18, 10]),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", ["primal", "dual"])
def test_reduced_operator_parity(ghb, name, kind):
    m, M = CASES[name]
    opts = {} if M is None else dict(M=tuple(M))
    ctx = ghb.Context.from_microstructure(m, **opts)
    assert ctx.M == [2 * n for n in m["N"]]
    ctx.set_form("reduced")
    op = OG.Operator(OC.material_from_dict(m), m["N"], kind, M=ctx.M)
    x = W.random_field(np.random.default_rng(len(name)), m["d"], m["N"])
    k = ghb.GHB_PRIMAL if kind == "primal" else ghb.GHB_DUAL
    for project in (True, False):
        ref = ghb.half_from_full(OG.reduced_matvec(x, op.a_M, kind if project else None))
        for dt, tol in [(torch.complex128, 1e-12), (torch.complex64, 2e-5)]:
            xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
            got = ctx.matvec(xt, kind=k, project=project).cpu().numpy()
            assert rel(got, ref) < tol, (name, kind, project, dt)


@pytest.mark.parametrize("N", [81, 2187])
def test_reduced_equals_double_grid_on_gpu(ghb, N):
    m = W.centred_disk(N, fraction=0.3, value=100.0)
    ctx = ghb.Context.from_microstructure(m)
    x = W.random_field(np.random.default_rng(N), 2, [N, N])
    for dt, tol in [(torch.complex128, 1e-12), (torch.complex64, 2e-5)]:
        xt = torch.from_numpy(np.ascontiguousarray(ghb.half_from_full(x))).to(dt).cuda()
        ctx.set_form("double_grid")
        a = ctx.matvec(xt).cpu().numpy()
        ctx.set_form("reduced")
        b = ctx.matvec(xt).cpu().numpy()
        assert rel(b, a) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-8)])
def test_reduced_bounds(ghb, precision, tol):
    m = W.random_disk_instance(9, N=45)
    ctx = ghb.Context.from_microstructure(m, precision=precision)
    U, L, _, _ = ctx.bounds()
    ctx.set_form("reduced")
    Ur, Lr, infos, st = ctx.bounds()
    assert st == 0 and rel(Ur, U) < tol and rel(Lr, L) < tol


def test_reduced_needs_m_2n(ghb):
    m = dict(d=2, N=[15, 15], a0=1.0, inclusions=[])
    ctx = ghb.Context.from_microstructure(m, M=(32, 30))
    with pytest.raises(ghb.GhbError):
        ctx.set_form("reduced")
