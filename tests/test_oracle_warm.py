"""Pins of the coarse-to-fine start and of the bounds along CG (Section 7.4).

* the prolongation is exact: the prolongated coefficients define the same
  trigonometric polynomial (point values by the defining sum) and, the Ga
  energies being exact integrals (Lemma integ_eval_VM), the same energy;
* a CG started from the prolongated coarse solution starts at the coarse
  bound, decreases monotonically and ends at the cold start's bound;
* the energies along CG follow J(e_i) = J(0) - sum_{j<i} alpha_j <r_j, r_j> from
  the CG scalars (checked against the energies evaluated by definition)."""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients as C
from oracle import galerkin as G


def _eval(x, pts):
    """sum_k x(k) exp(2 pi i k.p) at points p (d components)."""
    N = x.shape[1:]
    ks = C.freq_grid(list(N)).reshape(-1, len(N))
    ph = np.exp(2j * np.pi * pts @ ks.T)
    return np.array([ph @ x[c].reshape(-1) for c in range(x.shape[0])])


@pytest.mark.parametrize("Nc,Nf", [([5, 7], [11, 9]), ([3, 5, 3], [7, 5, 9])])
def test_prolongation_is_the_same_polynomial(Nc, Nf):
    rng = np.random.default_rng(len(Nc))
    d = len(Nc)
    x = rng.standard_normal((d,) + tuple(Nc)) + 1j * rng.standard_normal((d,) + tuple(Nc))
    pts = rng.uniform(-0.5, 0.5, (7, d))
    assert np.abs(_eval(G.prolong(x, Nf), pts) - _eval(x, pts)).max() < 1e-12 * np.abs(x).sum()


def test_prolongated_energy_and_warm_cg():
    N, Nc = 27, 9
    m = W.centred_disk(N, fraction=0.3, value=100.0)
    mat = C.material_from_dict(m)
    E = [1.0, 0.0]
    opc = G.Operator(mat, [Nc, Nc], G.PRIMAL)
    ec, _ = G.cg(opc, opc.rhs(E), 1e-12)
    Jc = opc.energy(G.constant_field(E, [Nc, Nc]) + ec, G.constant_field(E, [Nc, Nc]) + ec)
    op = G.Operator(mat, [N, N], G.PRIMAL)
    x0 = G.prolong(ec, [N, N])
    b = op.rhs(E)
    xw, infow = G.cg(op, b, 1e-10, x0=x0, track_energy_E=E)
    xz, infoz = G.cg(op, b, 1e-10, track_energy_E=E)
    ew, ez = np.array(infow["energies"]), np.array(infoz["energies"])
    assert abs(ew[0] - Jc) < 1e-12 * Jc                     # exact integration on both grids
    assert ez[0] == pytest.approx(mat.mean(), rel=1e-13)     # the Voigt start
    assert np.all(np.diff(ew) <= 1e-12 * Jc) and np.all(np.diff(ez) <= 1e-12 * ez[0])
    assert abs(ew[-1] - ez[-1]) < 1e-12 * ez[-1]


def test_energy_recurrence_matches_definition():
    """J(e_i) = J(0) - sum_{j<i} alpha_j <r_j, r_j> against the energies by definition."""
    N = 15
    m = dict(d=2, N=[N, N], a0=1.0, inclusions=[(0, (0, 0, 0), (2 ** -0.5, 2 ** -0.5, 1), 10.0)])
    mat = C.material_from_dict(m)
    E = [0.3, 1.0]
    op = G.Operator(mat, [N, N], G.PRIMAL)
    b = op.rhs(E)
    _, info = G.cg(op, b, 1e-12, track_energy_E=E)
    en = np.array(info["energies"])
    # the recurrence, written out with its own CG loop
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = G.inner(r, r)
    rec = [en[0]]
    dec = 0.0
    for _ in range(info["iters"]):
        q = op.apply(p)
        alpha = rr / G.inner(p, q)
        dec += alpha * rr
        rec.append(en[0] - dec)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = G.inner(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    assert np.abs(np.array(rec) - en).max() < 1e-12 * en[0]
