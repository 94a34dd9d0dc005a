"""GPU bounds at the measured families' sizes against stored oracle values
(tests/golden/*.json, written by tests/golden/make_golden.py from the CPU
oracle alone) and, at the full size N = 2187, against properties that hold at
any N (Löwner order of the bounds, monotone tightening in N from the stored
N = 729 values, square symmetry, Voigt/Reuss and Hashin-Shtrikman brackets).

Tolerances: FP64 path 1e-12 relative (the FP64 parity target); mixed path
1e-8 relative with the upper bound not below and the lower bound not above
the oracle by more than the one-sided slack of tests/conftest.py (1e-13)
relative.
"""
import json
import os

import numpy as np
import pytest

from conftest import one_sided_margins, one_sided_slack

import workloads as W
from oracle import coefficients as OC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ["square_N15", "disk_N81", "disk_N243", "disk_N729", "sphere_N33", "cube_N33"]


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


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_golden_bounds(ghb, name, prec):
    gd = load(name)
    m = gd["microstructure"]
    Uo, Lo = np.array(gd["upper"]), np.array(gd["lower"])
    ctx = ghb.Context.from_microstructure(m, precision=prec, tol=1e-11 if prec == "fp64" else 1e-10)
    U, L, infos, st = ctx.bounds()
    assert st == 0
    if prec == "fp64":
        assert rel(U, Uo) < 1e-12 and rel(L, Lo) < 1e-12
    else:
        assert rel(U, Uo) < 1e-8 and rel(L, Lo) < 1e-8
        su, sl = one_sided_slack(m)
        mu, ml = one_sided_margins(U, L, Uo, Lo)
        assert mu >= -su and ml >= -sl, (mu, ml, su, sl)


def _hs(a1, a2, f2, d):
    f1 = 1 - f2
    return a1 + f2 / (1 / (a2 - a1) + f1 / (d * a1)), a2 + f1 / (1 / (a1 - a2) + f2 / (d * a2))


def test_full_size_disk_properties(ghb):
    m = W.centred_disk(2187, fraction=0.3, value=100.0)
    ctx = ghb.Context.from_microstructure(m, precision="mixed", tol=1e-10)
    U, L, infos, st = ctx.bounds()
    assert st == 0
    g729 = load("disk_N729")
    U7, L7 = np.array(g729["upper"]), np.array(g729["lower"])
    assert np.all(np.linalg.eigvalsh(U7 - U) > -1e-12)       # eq. subspace_hierarchy
    assert np.all(np.linalg.eigvalsh(L - L7) > -1e-12)
    assert np.all(np.linalg.eigvalsh(U - L) > 0)             # Prop. struct_bounds
    assert abs(U[0, 1]) < 1e-9 * U[0, 0] and abs(U[0, 0] - U[1, 1]) < 1e-9 * U[0, 0]
    mat = OC.material_from_dict(m)
    lo, hi = _hs(1.0, 100.0, 0.3, 2)
    assert mat.harmonic_mean() < L[0, 0] <= U[0, 0] < mat.mean()
    assert U[0, 0] > lo and L[0, 0] < hi
    assert all(i["relres"] <= 1e-10 for i in infos)
