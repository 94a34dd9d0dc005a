"""Pins of the oracle's Ga operator, CG and bounds.

What fixes the answers here is the paper and the mathematics, not the oracle:
projection algebra (Def. projection, Lemma Helmholtz_decomp), brute force
with the dense Galerkin matrix (Lemma FD_matrix_full), dimensions of the
discrete spaces (Remark mem_req, Tab. memory), closed forms for a homogeneous
cell and for laminates, Voigt/Reuss and Hashin-Shtrikman bracketing, the bound
ordering and its monotonicity in N (Prop. struct_bounds, eq.
subspace_hierarchy), the Voigt start and monotone energies of CG (Section 7.4,
eq. minim_krylov) and the two-dimensional Keller duality.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import coefficients as C
from oracle import galerkin as G

rng0 = np.random.default_rng(20141206)


def disk_mat(a1=10.0, r=0.3, c=(0.0, 0.0), a0=1.0):
    return C.Material(2, a0, [C.Inclusion(C.DISK, c, (r,), a1)])


def rand_field(rng, d, N):
    return W.random_field(rng, d, N)


def test_projections_are_orthogonal_projections():
    for N in ([5, 7], [3, 5, 3]):
        GE = G.projection_matrices(N, G.PRIMAL)
        GJ = G.projection_matrices(N, G.DUAL)
        d = len(N)
        assert np.allclose(GE @ GE, GE, atol=1e-15)
        assert np.allclose(GJ @ GJ, GJ, atol=1e-15)
        assert np.allclose(GE @ GJ, 0, atol=1e-15)
        assert np.allclose(GE, np.swapaxes(GE, -1, -2))
        GU = np.zeros_like(GE)
        GU[tuple((n - 1) // 2 for n in N)] = np.eye(d)
        assert np.allclose(GE + GJ + GU, np.eye(d))


@pytest.mark.parametrize("N,Ms", [([5, 5], [[9, 9], [10, 12], [16, 16]]),
                                  ([7, 9], [[13, 17], [15, 18]]),
                                  ([3, 5, 3], [[5, 9, 5], [6, 10, 8]])])
@pytest.mark.parametrize("kind", [G.PRIMAL, G.DUAL])
def test_matvec_dense_equals_double_grid_any_M(N, Ms, kind):
    """Cor. Ga_linsys / Lemma integ_eval_VM: every M >= 2N-1 gives G A^full."""
    rng = np.random.default_rng(len(N) * 100 + N[0])
    d = len(N)
    incs = [C.Inclusion(C.BOX, (0.2, -0.1, 0.05), (0.5, 0.3, 0.4), 6.0)]
    mat = C.Material(d, 1.0, incs)
    x = rand_field(rng, d, N)
    ref = G.Operator(mat, N, kind, method="dense").apply(x)
    for M in Ms:
        got = G.Operator(mat, N, kind, M=M).apply(x)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    idx = np.array([[0] * d, [1] + [0] * (d - 1), [-(N[0] - 1) // 2] + [n // 2 for n in N[1:]]])
    samp = G.matvec_sampled(x, G.Operator(mat, N, kind, method="dense").mat, kind, idx)
    c = [(n - 1) // 2 for n in N]
    for s, l in enumerate(idx):
        assert np.abs(samp[s] - ref[(slice(None),) + tuple(l + c)]).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("N", [[5, 5], [5, 7], [3, 3, 3]])
def test_operator_rank_and_symmetry(N):
    """dim E_N = |N| - 1 and dim J_N = (d-1)(|N|-1) (Remark mem_req), and G A^full
    is self-adjoint and positive on the range of G (so G A^full G is Hermitian
    positive semi-definite with exactly that rank)."""
    d = len(N)
    n = int(np.prod(N))
    mat = C.Material(d, 1.0, [C.Inclusion(C.BOX, (0.0,) * 3, (0.5,) * 3, 3.0)])
    for kind, dim in ((G.PRIMAL, n - 1), (G.DUAL, (d - 1) * (n - 1))):
        op = G.Operator(mat, N, kind, method="dense")
        cols = []
        for j in range(d * n):
            e = np.zeros(d * n, dtype=complex)
            e[j] = 1
            cols.append(op.apply(G.project(e.reshape((d,) + tuple(N)), kind)).reshape(-1))
        K = np.array(cols).T
        assert np.allclose(K, K.conj().T, atol=1e-13)
        ev = np.linalg.eigvalsh(0.5 * (K + K.conj().T))
        assert np.sum(ev > 1e-10) == dim
        assert ev.min() > -1e-12


def test_cg_matches_dense_solve():
    mat = disk_mat(a1=20.0, r=0.25, c=(0.1, -0.07))
    for N in ([5, 5], [7, 5]):
        U1, L1, _ = G.bounds(mat, N, tol=1e-13)
        U2, L2, _ = G.bounds(mat, N, method="dense", op_method="dense")
        assert np.allclose(U1, U2, rtol=0, atol=1e-12 * np.abs(U2).max())
        assert np.allclose(L1, L2, rtol=0, atol=1e-12 * np.abs(L2).max())
    mat3 = C.Material(3, 1.0, [C.Inclusion(C.SPHERE, (0.05, 0, -0.1), (0.3,), 8.0)])
    U1, L1, _ = G.bounds(mat3, [3, 3, 3], tol=1e-13)
    U2, L2, _ = G.bounds(mat3, [3, 3, 3], method="dense", op_method="dense")
    assert np.allclose(U1, U2, rtol=0, atol=1e-12 * np.abs(U2).max())
    assert np.allclose(L1, L2, rtol=0, atol=1e-12 * np.abs(L2).max())


def test_homogeneous_cell_exact():
    for d in (2, 3):
        mat = C.Material(d, 3.7, [])
        U, L, infos = G.bounds(mat, [5] * d)
        assert np.allclose(U, 3.7 * np.eye(d), atol=1e-14)
        assert np.allclose(L, 3.7 * np.eye(d), atol=1e-14)
        assert all(i["iters"] == 0 for i in infos.values())


@pytest.mark.parametrize("d", [2, 3])
def test_laminate_closed_forms(d):
    """Layers normal to e1: along the layers the upper bound is the arithmetic
    mean and across them the lower bound is the harmonic mean, exactly, at every
    N (the exact minimisers e = 0, j = 0 lie in the discrete spaces)."""
    m = W.laminate(5, d=d, h=0.37, value=8.0, a0=1.5, center=0.11)
    mat = C.material_from_dict(m)
    arith = 1.5 + (8.0 - 1.5) * 0.37
    harm = 1.0 / (1 / 1.5 + (1 / 8.0 - 1 / 1.5) * 0.37)
    prev = None
    for N in (3, 5, 7, 9):
        U, L, _ = G.bounds(mat, [N] * d, tol=1e-13)
        for a in range(1, d):
            assert abs(U[a, a] - arith) < 1e-13
        assert abs(L[0, 0] - harm) < 1e-13
        off = U - np.diag(np.diag(U))
        assert np.abs(off).max() < 1e-13
        assert harm - 1e-13 <= U[0, 0] <= arith and harm <= L[1, 1] <= arith + 1e-13
        if prev is not None:
            assert U[0, 0] <= prev[0] + 1e-13 and L[1, 1] >= prev[1] - 1e-13
        prev = (U[0, 0], L[1, 1])


def _hs(a1, a2, f2, d):
    """Hashin-Shtrikman bounds for two isotropic phases (matrix a1, inclusion a2 > a1)."""
    f1 = 1 - f2
    lo = a1 + f2 / (1 / (a2 - a1) + f1 / (d * a1))
    hi = a2 + f1 / (1 / (a1 - a2) + f2 / (d * a2))
    return lo, hi


def test_config1_square_bracketing_and_symmetry():
    """d = 2 centred square (volume fraction 1/2, contrast 10): square symmetry
    makes both bounds multiples of I; Reuss <= HS- ... ordering holds."""
    m = W.centred_square(15)
    mat = C.material_from_dict(m)
    U, L, infos = G.bounds(mat, m["N"], tol=1e-10)
    assert np.abs(U - U[0, 0] * np.eye(2)).max() < 1e-9 * U[0, 0]
    assert np.abs(L - L[0, 0] * np.eye(2)).max() < 1e-9 * L[0, 0]
    voigt, reuss = mat.mean(), mat.harmonic_mean()
    lo, hi = _hs(1.0, 10.0, 0.5, 2)
    assert reuss < L[0, 0] < U[0, 0] < voigt
    assert U[0, 0] > lo and L[0, 0] < hi
    # M = 2N - 1 (prime 29) and the 5-smooth M = 30 give the same bounds
    U30, L30, _ = G.bounds(mat, m["N"], M=[30, 30], tol=1e-10)
    assert np.allclose(U30, U, rtol=1e-9) and np.allclose(L30, L, rtol=1e-9)


def test_disk_hs_and_monotone_in_N():
    mat = C.material_from_dict(W.centred_disk(5, value=100.0))
    f2 = 0.3
    lo, hi = _hs(1.0, 100.0, f2, 2)
    prevU = prevL = None
    for N in (5, 9, 15, 21):
        U, L, _ = G.bounds(mat, [N, N], tol=1e-11)
        assert np.all(np.linalg.eigvalsh(U - L) > 0)
        assert U[0, 0] > lo and L[0, 0] < hi
        if prevU is not None:   # eq. subspace_hierarchy: nested spaces
            assert np.all(np.linalg.eigvalsh(prevU - U) > -1e-10)
            assert np.all(np.linalg.eigvalsh(L - prevL) > -1e-10)
        prevU, prevL = U, L


def test_cg_voigt_start_and_monotone_energy():
    """Section 7.4: from x0 = 0 the first bound is the Voigt mean <A>E.E, and CG
    (a Krylov minimisation, eq. minim_krylov) never increases the energy."""
    mat = C.material_from_dict(W.centred_square(9, side=0.8, value=1e4))
    op = G.Operator(mat, [9, 9], G.PRIMAL)
    E = np.array([1.0, 0.0])
    _, info = G.cg(op, op.rhs(E), tol=1e-10, track_energy_E=E)
    en = np.array(info["energies"])
    assert abs(en[0] - mat.mean()) < 1e-9 * mat.mean()
    assert np.all(np.diff(en) <= 1e-9 * en[0])
    assert en[-1] < 0.5 * en[0]


def test_keller_duality_2d():
    """R (90 degree rotation) maps E_N onto J_N and the table of 1/a equals that
    of the phase-swapped material over a1 a2, so D(a1, a2) = R^T U(a2, a1) R / (a1 a2)."""
    a1, a2 = 2.0, 13.0
    c = (0.13, -0.21)
    mat = C.Material(2, a1, [C.Inclusion(C.DISK, c, (0.27,), a2)])
    swp = C.Material(2, a2, [C.Inclusion(C.DISK, c, (0.27,), a1)])
    N = [9, 9]
    _, L, _ = G.bounds(mat, N, tol=1e-12)
    Us, _, _ = G.bounds(swp, N, tol=1e-12)
    R = np.array([[0.0, -1.0], [1.0, 0.0]])
    D = np.linalg.inv(L)
    assert np.allclose(D, R.T @ Us @ R / (a1 * a2), rtol=1e-10, atol=1e-12)


def test_sphere_bounds_3d_small():
    mat = C.material_from_dict(W.centred_sphere(5, value=50.0))
    U, L, _ = G.bounds(mat, [5, 5, 5], tol=1e-11)
    lo, hi = _hs(1.0, 50.0, 0.2, 3)
    assert np.all(np.linalg.eigvalsh(U - L) > 0)
    assert U[0, 0] > lo and L[0, 0] < hi
    assert np.abs(U - U[0, 0] * np.eye(3)).max() < 1e-9 * U[0, 0]    # cubic symmetry
    assert mat.harmonic_mean() < L[0, 0] and U[0, 0] < mat.mean()


@pytest.mark.parametrize("d,kind", [(2, "primal"), (2, "dual"), (3, "primal"), (3, "dual")])
def test_admissible_projection(d, kind):
    """The nearest admissible fluctuation (Def. trig_pol, Def. projection):
    identity on admissible fields, idempotent, Hermitian and in the range of G;
    on a perturbed admissible field it removes exactly the perturbation's
    non-Hermitian and out-of-range parts."""
    rng = np.random.default_rng(17 + d)
    N = [7, 9] if d == 2 else [5, 7, 3]
    x = W.random_field(rng, d, N, hermitian=False)
    a = G.admissible(x, kind)
    flip = a[(slice(None),) + (slice(None, None, -1),) * d]
    assert np.abs(a - np.conj(flip)).max() < 1e-14 * np.abs(a).max()          # Hermitian
    assert np.abs(G.project(a, kind) - a).max() < 1e-14 * np.abs(a).max()      # in range(G)
    assert np.abs(G.admissible(a, kind) - a).max() < 1e-14 * np.abs(a).max()  # idempotent
    h = G.project(W.random_field(rng, d, N), kind)                              # admissible
    assert np.abs(G.admissible(h, kind) - h).max() < 1e-14 * np.abs(h).max()
    # the removed part is orthogonal to every admissible field
    r = x - a
    assert abs(G.inner(r, h)) < 1e-12 * np.sqrt(G.inner(r, r) * G.inner(h, h))
