"""GPU bounds at the measured families' full sizes against stored oracle values
(tests/golden/*.json, written by tests/golden/make_golden.py from the CPU
oracle alone; Def. Ga, eq. GA_prim, Prop. struct_bounds):

* d = 2 centred disk, contrast 100, N = 2187 (M = 4374): the bench workload;
* d = 3 centred sphere (volume fraction 0.2) and cube (side 0.6), contrast
  1000, N = 65 (M = 135);
* the largest-contrast instance (about 1e4) of the 512-instance disk batch at
  N = 255, through a context and through the batch engine;
* d = 3 sphere and cube at N = 129 (M = 270): the bounds of the 24th CG
  iterate (a converged oracle solve takes hours there), against the FP64 path
  capped at 24 iterations; the converged mixed bounds must lie inside both the
  24-iterate bounds and the N = 65 bounds (the spaces grow with N, so the
  bounds tighten, eq. subspace_hierarchy).

Tolerances: FP64 path 1e-12 relative, mixed path 1e-8 relative with the
one-sided slack of tests/conftest.py.
"""
import json
import os

import numpy as np
import pytest

from conftest import one_sided_margins, one_sided_slack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def check(U, L, gd, prec):
    m = gd["microstructure"]
    Uo, Lo = np.array(gd["upper"]), np.array(gd["lower"])
    if prec == "fp64":
        assert rel(U, Uo) < 1e-12 and rel(L, Lo) < 1e-12, (rel(U, Uo), rel(L, Lo))
    else:
        assert rel(U, Uo) < 1e-8 and rel(L, Lo) < 1e-8, (rel(U, Uo), rel(L, Lo))
        mu, ml = one_sided_margins(U, L, Uo, Lo)
        su, sl = one_sided_slack(m)
        assert mu >= -su and ml >= -sl, (mu, ml, su, sl)


@pytest.mark.parametrize("name", ["disk_N2187", "sphere_N65", "cube_N65", "batch_maxcontrast_N255"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fullsize_golden(ghb, name, prec):
    gd = load(name)
    m = gd["microstructure"]
    ctx = ghb.Context.from_microstructure(m, precision=prec, tol=1e-11 if prec == "fp64" else 1e-10)
    U, L, infos, st = ctx.bounds()
    assert st == 0
    check(U, L, gd, prec)
    ctx.close()


def test_batch_engine_high_contrast(ghb):
    """The same high-contrast instance through the batch engine (mixed
    precision, batched CUDA-graph iterations) beside two other requests."""
    import workloads as W
    gd = load("batch_maxcontrast_N255")
    b = ghb.Batch()
    tid = b.submit(gd["microstructure"])
    b.submit(W.random_disk_instance(W.BASE_SEED + 3, N=101))
    b.submit(W.random_disk_instance(W.BASE_SEED + 4, N=47))
    b.run(iterations=8)
    r = {x["id"]: x for x in b.results()}[tid]
    b.close()
    assert r["status"] == 0
    check(r["upper"], r["lower"], gd, "mixed")


@pytest.mark.parametrize("shape", ["sphere", "cube"])
def test_fixed_iterations_N129(ghb, shape):
    """The FP64 path capped at the golden's 24 CG iterations reports
    GHB_ERR_NOT_CONVERGED and gives the oracle's bounds of the 24th iterate."""
    gd = load(f"{shape}_N129_k24")
    m = gd["microstructure"]
    K = gd["maxiter"]
    ctx = ghb.Context.from_microstructure(m, precision="fp64", tol=1e-30, max_iter=K, M=tuple(gd["M"]))
    U, L, infos, st = ctx.bounds()
    assert st == ghb.GHB_ERR_NOT_CONVERGED
    assert all(i["iters"] == K and i["status"] == ghb.GHB_ERR_NOT_CONVERGED for i in infos)
    assert rel(U, gd["upper"]) < 1e-12 and rel(L, gd["lower"]) < 1e-12, (rel(U, gd["upper"]), rel(L, gd["lower"]))
    ctx.close()


@pytest.mark.parametrize("shape", ["sphere", "cube"])
def test_mixed_N129_inside_coarser_bounds(ghb, shape):
    """Converged mixed bounds at N = 129 (M = 270, the size-specialised
    passes) lie inside the oracle's 24-iterate bounds at N = 129 and inside its
    converged bounds at N = 65, and lower <= upper (Prop. struct_bounds)."""
    g129 = load(f"{shape}_N129_k24")
    g65 = load(f"{shape}_N65")
    m = g129["microstructure"]
    ctx = ghb.Context.from_microstructure(m, precision="mixed", tol=1e-10)
    assert ctx.M == [270, 270, 270]
    U, L, infos, st = ctx.bounds()
    assert st == 0
    su, sl = one_sided_slack(m)
    for gd in (g129, g65):
        Uo, Lo = np.array(gd["upper"]), np.array(gd["lower"])
        assert np.all(np.linalg.eigvalsh(Uo - U) > -su * np.abs(Uo).max())
        assert np.all(np.linalg.eigvalsh(L - Lo) > -sl * np.abs(Lo).max())
    assert np.all(np.linalg.eigvalsh(U - L) > 0)
    ctx.close()
