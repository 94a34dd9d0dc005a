"""Failure statuses of the solves, reached from the host with valid inputs.

* GHB_ERR_NOT_CONVERGED: a cap on the CG iterations.  The outputs are still
  filled and are still guaranteed bounds (Def. Ga: the energy of any admissible
  field is an upper bound, eq. spd_inverse_ineq for the dual): the capped upper
  bound dominates the converged oracle's in the Löwner order and the capped
  lower bound is dominated by it.  The FP64 path capped at K iterations gives
  the oracle's bounds of its K-th iterate.
* GHB_ERR_BREAKDOWN: an inclusion value that is finite in FP64 but overflows
  FP32 (1e39) makes the FP32 inner operator non-finite, so the first curvature
  <p, Ap> of the inner CG is not finite; the mixed solve stops with
  GHB_ERR_BREAKDOWN and the context stays usable.
No GPU fault, trap or hang is involved: both are arithmetic outcomes that the
solver checks on the device and reports through its state.
"""
import numpy as np
import pytest

from conftest import one_sided_slack

from oracle import coefficients as OC
from oracle import galerkin as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = dict(d=2, N=[45, 31], a0=1.0, inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 100.0)])


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_not_converged_bounds_are_guaranteed(ghb, prec):
    mat = OC.material_from_dict(SPEC)
    ctx = ghb.Context.from_microstructure(SPEC, precision=prec, max_iter=3)
    U, L, infos, st = ctx.bounds()
    assert st == ghb.GHB_ERR_NOT_CONVERGED
    assert all(i["status"] == ghb.GHB_ERR_NOT_CONVERGED for i in infos)
    assert all(i["relres"] > 1e-10 for i in infos)
    Uo, Lo, _ = OG.bounds(mat, SPEC["N"], M=ctx.M, tol=1e-12)
    su, sl = one_sided_slack(SPEC)
    assert np.all(np.linalg.eigvalsh(U - Uo) > -su * np.abs(Uo).max())
    assert np.all(np.linalg.eigvalsh(Lo - L) > -sl * np.abs(Lo).max())
    assert np.all(np.linalg.eigvalsh(U - L) > 0)
    assert rel(U, Uo) > 1e-6        # three iterations are far from the minimiser
    if prec == "fp64":
        assert all(i["iters"] == 3 for i in infos)
        U3, L3, _ = OG.bounds(mat, SPEC["N"], M=ctx.M, tol=1e-30, maxiter=3)
        assert rel(U, U3) < 1e-12 and rel(L, L3) < 1e-12
    ctx.close()


def test_breakdown_reported_and_context_usable(ghb):
    bad = dict(SPEC, inclusions=[(1, (0.05, 0.1, 0), (0.3, 0, 0), 1e39)])
    ctx = ghb.Context.from_microstructure(bad, precision="mixed")
    with pytest.raises(ghb.GhbError) as err:
        ctx.bounds()
    assert err.value.status == ghb.GHB_ERR_BREAKDOWN
    # the same context with an ordinary material afterwards
    ctx.set_coeffs(SPEC["a0"], SPEC["inclusions"])
    U, L, infos, st = ctx.bounds()
    assert st == 0
    Uo, Lo, _ = OG.bounds(OC.material_from_dict(SPEC), SPEC["N"], M=ctx.M, tol=1e-12)
    assert rel(U, Uo) < 1e-8 and rel(L, Lo) < 1e-8
    ctx.close()
