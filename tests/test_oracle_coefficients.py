"""Pins of the oracle's coefficient tables (Remark anal_Fourier, eq. char_func_Four,
eq. inclcomp_formula, Lemma integ_eval_VM).

Each shape coefficient is checked against numerical quadrature of its defining
integral f^(k) = int_Y f(x) exp(-2 pi i k.x) dx (Section 2.2), the shift sign
against a direct 2-D quadrature of an off-centre disk, and the double-grid
values against the bilinear form they must reproduce.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import j0

from oracle import coefficients as C
from oracle import fourier as F
from oracle import galerkin as G


@pytest.mark.parametrize("k", [(0, 0), (1, 0), (2, 3), (-5, 4)])
def test_box_coefficient_quadrature(k):
    h = (0.37, 0.81)
    ref = 1.0
    for a in range(2):
        re = integrate.quad(lambda x: math.cos(2 * math.pi * k[a] * x), -h[a] / 2, h[a] / 2)[0]
        ref *= re                       # the centred box is even: imaginary part 0
    got = C.shape_coeff(C.BOX, np.array([k]), h)[0]
    assert abs(got - ref) < 1e-12


@pytest.mark.parametrize("k", [(0, 0), (1, 0), (3, 4), (-7, 2), (20, 13)])
def test_disk_coefficient_hankel(k):
    """Radial transform in 2-D: F(rho) = 2 pi int_0^r s J0(2 pi rho s) ds."""
    r = 0.3090194
    rho = math.hypot(*k)
    ref = integrate.quad(lambda s: 2 * math.pi * s * j0(2 * math.pi * rho * s), 0, r, epsabs=1e-14, limit=200)[0]
    got = C.shape_coeff(C.DISK, np.array([k]), (r,))[0]
    assert abs(got - ref) < 1e-11


@pytest.mark.parametrize("k", [(0, 0, 0), (0, 0, 1), (1, 2, 2), (5, -3, 7), (0.001, 0, 0)])
def test_sphere_coefficient_radial(k):
    """Radial transform in 3-D: F(rho) = 4 pi int_0^r s^2 sin(2 pi rho s)/(2 pi rho s) ds."""
    r = 0.3627832
    rho = math.sqrt(sum(v * v for v in k))

    def f(s):
        q = 2 * math.pi * rho * s
        return 4 * math.pi * s * s * (math.sin(q) / q if q > 0 else 1.0)
    ref = integrate.quad(f, 0, r, epsabs=1e-15, limit=200)[0]
    got = C.shape_coeff(C.SPHERE, np.array([k], dtype=float), (r,))[0]
    assert abs(got - ref) < 1e-12


def test_sphere_fraction_radius():
    r = (3 * 0.2 / (4 * math.pi)) ** (1 / 3)
    assert abs(r - 0.3627832) < 1e-7
    assert abs(C.shape_coeff(C.SPHERE, np.zeros((1, 3)), (r,))[0] - 0.2) < 1e-14


@pytest.mark.parametrize("k", [(1, 0), (2, -3)])
def test_shift_sign_offcentre_disk(k):
    """f(x - x_i) has coefficient exp(-2 pi i k.x_i) f^(k): checked by a direct
    2-D quadrature over the shifted disk (polar coordinates around x_i)."""
    c = np.array([0.17, -0.23])
    r = 0.2
    mat = C.Material(2, 0.0, [C.Inclusion(C.DISK, tuple(c), (r,), 1.0)])

    def integrand(t, s, part):
        x = c + s * np.array([math.cos(t), math.sin(t)])
        ph = -2 * math.pi * (k[0] * x[0] + k[1] * x[1])
        return s * (math.cos(ph) if part == 0 else math.sin(ph))
    re = integrate.dblquad(lambda t, s: integrand(t, s, 0), 0, r, 0, 2 * math.pi, epsabs=1e-13)[0]
    im = integrate.dblquad(lambda t, s: integrand(t, s, 1), 0, r, 0, 2 * math.pi, epsabs=1e-13)[0]
    got = C.coeff_at(mat, np.array([k]))[0]
    assert abs(got - complex(re, im)) < 1e-10


def test_table_hermitian_and_mean():
    mat = C.Material(2, 2.0, [C.Inclusion(C.DISK, (0.1, 0.2), (0.2,), 7.0),
                              C.Inclusion(C.BOX, (-0.3, -0.25), (0.2, 0.3), 0.5)])
    t = C.coeff_table(mat, [9, 9])
    assert np.allclose(t, np.conj(t[::-1, ::-1]), atol=1e-15)      # real coefficient
    f1 = math.pi * 0.04
    f2 = 0.06
    assert abs(t[8, 8] - (2.0 + 5.0 * f1 - 1.5 * f2)) < 1e-14        # a^(0) = <a>
    assert abs(mat.mean() - (2.0 + 5.0 * f1 - 1.5 * f2)) < 1e-14


def _bilinear_dense(table, u, v):
    """sum_{k,l} a^(l-k) u(k) conj(v(l)) -- the form of Lemma FD_matrix_full."""
    A = G.dense_galerkin(table, u.shape)
    return np.vdot(v.reshape(-1), A @ u.reshape(-1))


@pytest.mark.parametrize("N,M", [((5, 5), (9, 9)), ((5, 7), (9, 14)), ((7, 7), (16, 15)),
                                 ((3, 5, 3), (5, 9, 6))])
def test_double_grid_quadrature_is_exact(N, M):
    """Lemma integ_eval_VM: for M >= 2N-1, (1/|M|) sum_m A_M(x_m) u(x_m) v(x_m)
    equals the exact integral sum_{k,l} a^(l-k) u^(k) conj(v^(l))."""
    rng = np.random.default_rng(sum(N) + sum(M))
    d = len(N)
    incs = [C.Inclusion(C.BOX, tuple(rng.uniform(-0.5, 0.5, 3)), tuple(rng.uniform(0.1, 0.6, 3)), 4.0)]
    if d == 2:
        incs.append(C.Inclusion(C.DISK, (0.3, -0.2, 0), (0.15,), 9.0))
    mat = C.Material(d, 1.5, incs)
    table = C.coeff_table(mat, N)
    aM = G.double_grid_values(table, M)
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    uM = F.idft_nd(F.pad_centred_to_wrapped(u, M), axes=range(d))
    vM = F.idft_nd(F.pad_centred_to_wrapped(v, M), axes=range(d))
    quad = np.sum(aM * uM * np.conj(vM)) / np.prod(M)
    assert abs(quad - _bilinear_dense(table, u, v)) < 1e-12 * np.abs(table).sum() * np.abs(u).sum()
    assert np.abs(np.imag(G.double_grid_values(table, M))).max() == 0


def test_double_grid_too_coarse_aliases():
    """A grid M = 2N-3 violates the lemma's hypothesis and the quadrature is no
    longer exact (the bound on M is sharp), so a wrong M is caught."""
    rng = np.random.default_rng(3)
    N, M = (7, 7), (11, 11)
    mat = C.Material(2, 1.0, [C.Inclusion(C.DISK, (0.1, 0.05), (0.3,), 10.0)])
    table = C.coeff_table(mat, N)
    padded = F.pad_centred_to_wrapped(table[1:-1, 1:-1], M)          # Z_{2N-3} part only
    aM = F.idft_nd(padded, axes=range(2)).real
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    uM = F.idft_nd(F.pad_centred_to_wrapped(u, M), axes=range(2))
    quad = np.sum(aM * uM * np.conj(uM)) / np.prod(M)
    assert abs(quad - _bilinear_dense(table, u, u)) > 1e-6


def test_validate_rejects_bad_inputs():
    with pytest.raises(ValueError):
        C.validate(C.Material(2, -1.0, []))
    with pytest.raises(ValueError):
        C.validate(C.Material(2, 1.0, [C.Inclusion(C.DISK, (0, 0), (0.6,), 2.0)]))
    with pytest.raises(ValueError):   # overlapping through the periodic boundary
        C.validate(C.Material(2, 1.0, [C.Inclusion(C.DISK, (0.45, 0), (0.1,), 2.0),
                                       C.Inclusion(C.DISK, (-0.45, 0), (0.1,), 2.0)]))


def test_validate_overlap_every_pair():
    """Every pair of inclusions is checked, boxes included, through the
    periodic boundary; touching shapes are allowed (their open interiors are
    disjoint, so the table of 1/a is still of the composite form)."""
    B, D, S = C.BOX, C.DISK, C.SPHERE
    bad = [
        [C.Inclusion(B, (0.45, 0.0), (0.2, 0.2), 2.0), C.Inclusion(B, (-0.45, 0.05), (0.2, 0.2), 3.0)],
        [C.Inclusion(B, (0.0, 0.0), (0.4, 0.4), 2.0), C.Inclusion(D, (0.3, 0.3), (0.15,), 3.0)],
        [C.Inclusion(D, (0.3, 0.3), (0.15,), 3.0), C.Inclusion(B, (0.0, 0.0), (0.4, 0.4), 2.0)],
        [C.Inclusion(B, (0.0, 0.45), (1.0, 0.3), 2.0), C.Inclusion(D, (0.3, -0.4), (0.1,), 3.0)],
    ]
    for incs in bad:
        with pytest.raises(ValueError):
            C.validate(C.Material(2, 1.0, incs))
    good = [
        [C.Inclusion(B, (0.45, 0.0), (0.2, 0.2), 2.0), C.Inclusion(B, (-0.2, 0.0), (0.2, 0.2), 3.0)],
        [C.Inclusion(B, (0.0, 0.0), (0.4, 0.4), 2.0), C.Inclusion(D, (0.3, 0.3), (0.1,), 3.0)],
        [C.Inclusion(B, (0.0, 0.0), (0.4, 0.4), 2.0), C.Inclusion(B, (0.4, 0.0), (0.4, 0.4), 3.0)],  # touching
    ]
    for incs in good:
        C.validate(C.Material(2, 1.0, incs))
    with pytest.raises(ValueError):   # 3-D: a sphere meeting a box through the z boundary
        C.validate(C.Material(3, 1.0, [C.Inclusion(B, (0.0, 0.0, 0.45), (0.3, 0.3, 0.2), 2.0),
                                       C.Inclusion(S, (0.0, 0.0, -0.35), (0.1,), 3.0)]))
    C.validate(C.Material(3, 1.0, [C.Inclusion(B, (0.0, 0.0, 0.45), (0.3, 0.3, 0.2), 2.0),
                                   C.Inclusion(S, (0.0, 0.0, -0.2), (0.1,), 3.0)]))


def test_validate_overlap_against_sampled_shapes():
    """Brute force: random pairs of boxes and disks, overlap decided by
    sampling the two periodic characteristic functions on a 512^2 point grid;
    pairs within two grid spacings of touching are skipped (undecidable by
    sampling).  The validation must agree on every other pair."""
    rng = np.random.default_rng(4)
    n = 512
    x = (np.arange(n) + 0.5) / n - 0.5
    X, Y = np.meshgrid(x, x, indexing="ij")

    def inside(inc, margin):
        dx = X - inc.center[0]
        dy = Y - inc.center[1]
        dx -= np.round(dx)
        dy -= np.round(dy)
        if inc.shape == C.BOX:
            return (np.abs(dx) < 0.5 * inc.size[0] - margin) & (np.abs(dy) < 0.5 * inc.size[1] - margin)
        return np.hypot(dx, dy) < inc.size[0] - margin

    h = 2.0 / n
    checked = 0
    for _ in range(300):
        incs = []
        for _k in range(2):
            c = tuple(rng.uniform(-0.5, 0.5, 2))
            if rng.uniform() < 0.5:
                incs.append(C.Inclusion(C.BOX, c, tuple(rng.uniform(0.05, 0.5, 2)), 2.0))
            else:
                incs.append(C.Inclusion(C.DISK, c, (rng.uniform(0.03, 0.25),), 2.0))
        surely = np.any(inside(incs[0], 0.0) & inside(incs[1], h))          # a point well inside both
        maybe = np.any(inside(incs[0], -h) & inside(incs[1], -h))           # grown shapes meet
        if surely == maybe:
            try:
                C.validate(C.Material(2, 1.0, incs))
                rejected = False
            except ValueError:
                rejected = True
            assert rejected == bool(surely), incs
            checked += 1
    assert checked > 200


def test_inner_exact_sums_without_cancellation_loss():
    """The bound energies' scalar product: products rounded once, their sum
    exact up to the last rounding (Shewchuk's summation, math.fsum)."""
    from oracle import galerkin as G
    x = np.array([1e16, 1.0, -1e16, 3.0 + 2.0j])
    y = np.array([1.0, 1.0, 1.0, 1.0 - 1.0j])
    assert G.inner_exact(x, y) == 1.0 + 3.0 - 2.0
    rng = np.random.default_rng(0)
    a = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    b = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    assert abs(G.inner_exact(a, b) - G.inner(a, b)) < 1e-12 * np.abs(a).sum()


def test_large_argument_accuracy_against_mpmath():
    """High frequencies (N up to 2187 reaches |n| ~ 3000): the sinc factor, the
    disk's J1 term and the shift phase against 30-digit mpmath evaluations."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    h = 0.7071067811865476
    for k in [1, 37, 999, 2186, 3001]:
        ref = float(mpmath.sin(mpmath.pi * h * k) / (mpmath.pi * h * k)) * h
        got = C.shape_coeff(C.BOX, np.array([[k, 0]]), (h, 1.0))[0].real
        assert abs(got - ref) < 1e-16 + 1e-15 * abs(ref) + 1e-15 / k
    r = 0.3090194
    for k in [(3, 4), (700, 11), (2186, 2186), (1500, -900)]:
        rho = mpmath.sqrt(k[0] ** 2 + k[1] ** 2)
        ref = float(r * mpmath.besselj(1, 2 * mpmath.pi * r * rho) / rho)
        got = C.shape_coeff(C.DISK, np.array([k]), (r,))[0].real
        # FP64 rounds the argument x = 2 pi r |k| by about x eps, which moves the
        # oscillating J1 by up to |J1'| x eps ~ envelope * x eps
        x = 2 * math.pi * r * float(rho)
        env = r / float(rho) * math.sqrt(2 / (math.pi * x))
        assert abs(got - ref) < env * (x * 4e-16 + 1e-15)
    c = (0.1234567891, -0.3141592653)
    mat = C.Material(2, 0.0, [C.Inclusion(C.BOX, c, (1.0, 1.0), 1.0)])   # full cell: f^ = delta
    for k in [(0, 0)]:
        assert abs(C.coeff_at(mat, np.array([k]))[0] - 1.0) < 1e-15
    mat = C.Material(2, 0.0, [C.Inclusion(C.DISK, c, (r,), 1.0)])
    for k in [(2186, 1093), (-3000, 17)]:
        t = mpmath.mpf(k[0]) * mpmath.mpf(c[0]) + mpmath.mpf(k[1]) * mpmath.mpf(c[1])
        ph = complex(mpmath.exp(-2j * mpmath.pi * t))
        rho = mpmath.sqrt(k[0] ** 2 + k[1] ** 2)
        f = float(r * mpmath.besselj(1, 2 * mpmath.pi * r * rho) / rho)
        got = C.coeff_at(mat, np.array([k]))[0]
        x = 2 * math.pi * r * float(rho)
        env = r / float(rho) * math.sqrt(2 / (math.pi * x))
        assert abs(got - ph * f) < env * (x * 4e-16 + 1e-14)
