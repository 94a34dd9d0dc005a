"""Pins of the oracle's GaNi scheme (Def. GaNi, Algorithm 1, eq. GaNi_apost).

* brute force: the GaNi operator equals the periodic convolution with the
  discrete Fourier coefficients of the samples, (A~ x)(l) = sum_k a~((l-k) mod N) x(k)
  with a~(m) = (1/|N|) sum_j a(x^j) exp(-2 pi i m.x^j), assembled by loops;
* homogeneous material: every matrix is a0 I;
* laminate: the GaNi matrices are the arithmetic mean of the samples along the
  layers and their harmonic mean across (closed form of the discrete problem),
  and the a-posteriori bounds bracket the continuous laminate's A_H
  (arithmetic / harmonic means of a);
* duality for odd N (Remark duality_gani): B~_N^{-1} = A~_N;
* optimality of Ga: the Ga bounds lie inside the a-posteriori GaNi bounds.
"""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import coefficients as C
from oracle import galerkin as G
from oracle import gani as GN


def test_samples_point_rule():
    """Point membership on a 5 x 5 grid: a centred box of side 0.4 holds the
    points with |k/5 wrapped| <= 0.2, i.e. k in {0, 1, 4} per axis."""
    mat = C.Material(2, 1.0, [C.Inclusion(C.BOX, (0.0, 0.0), (0.4, 0.4), 3.0)])
    s = GN.sample_values(mat, [5, 5])
    inside = np.zeros((5, 5), dtype=bool)
    for i, j in itertools.product([0, 1, 4], repeat=2):
        inside[i, j] = True
    assert np.array_equal(s == 3.0, inside) and np.all(s[~inside] == 1.0)
    # a disk of radius 0.3 around (0.4, 0): points within periodic distance 0.3
    mat = C.Material(2, 2.0, [C.Inclusion(C.DISK, (0.4, 0.0), (0.3,), 7.0)])
    s = GN.sample_values(mat, [5, 5])
    for i, j in itertools.product(range(5), repeat=2):
        dx = (i / 5 - 0.4 + 0.5) % 1.0 - 0.5
        dy = (j / 5 + 0.5) % 1.0 - 0.5
        assert (s[i, j] == 7.0) == (dx * dx + dy * dy <= 0.09 + 1e-15)


@pytest.mark.parametrize("N", [[5, 5], [7, 3], [3, 5, 3]])
def test_operator_brute_force(N):
    rng = np.random.default_rng(sum(N))
    d = len(N)
    incs = [C.Inclusion(C.BOX, tuple(rng.uniform(-0.5, 0.5, 3)), tuple(rng.uniform(0.2, 0.7, 3)), 4.0)]
    mat = C.Material(d, 1.5, incs)
    op = GN.GaNiOperator(mat, N, G.PRIMAL)
    a = GN.sample_values(mat, N)
    n = int(np.prod(N))
    pts = list(itertools.product(*[range(v) for v in N]))               # grid index j
    freqs = list(itertools.product(*[range(-(v - 1) // 2, (v - 1) // 2 + 1) for v in N]))   # centred k
    atil = {}
    for m in itertools.product(*[range(v) for v in N]):                 # m mod N
        s = 0.0
        for j in pts:
            s += a[j] * np.exp(-2j * np.pi * sum(m[t] * j[t] / N[t] for t in range(d)))
        atil[m] = s / n
    x = rng.standard_normal((d,) + tuple(N)) + 1j * rng.standard_normal((d,) + tuple(N))
    y = np.zeros_like(x)
    cen = [(v - 1) // 2 for v in N]
    for li, l in enumerate(freqs):
        for ki, k in enumerate(freqs):
            m = tuple((l[t] - k[t]) % N[t] for t in range(d))
            y[(slice(None),) + tuple(l[t] + cen[t] for t in range(d))] += \
                atil[m] * x[(slice(None),) + tuple(k[t] + cen[t] for t in range(d))]
    got = op.apply(x, project_out=False)
    assert np.abs(got - y).max() < 1e-12 * np.abs(y).max()


def test_homogeneous():
    mat = C.Material(2, 3.5, [])
    up, lo, A, Binv, _ = GN.gani_bounds(mat, [7, 7])
    for X in (up, lo, A, Binv):
        assert np.abs(X - 3.5 * np.eye(2)).max() < 1e-13


@pytest.mark.parametrize("N", [9, 15])
def test_laminate_closed_forms(N):
    m = W.laminate(N, d=2, h=0.37, value=8.0, a0=1.0, center=0.05)
    mat = C.material_from_dict(m)
    s = GN.sample_values(mat, [N, N])
    col = s[:, 0]                                   # the samples vary along axis 0 only
    assert np.all(s == col[:, None])
    up, lo, A, Binv, _ = GN.gani_bounds(mat, [N, N])
    harm_s, arith_s = 1.0 / np.mean(1.0 / col), np.mean(col)
    assert abs(A[0, 0] - harm_s) < 1e-10 * arith_s and abs(A[1, 1] - arith_s) < 1e-10 * arith_s
    assert abs(A[0, 1]) < 1e-10 * arith_s
    assert np.abs(Binv - A).max() < 1e-10 * arith_s
    harm, arith = mat.harmonic_mean(), mat.mean()     # the continuous laminate's A_H
    assert lo[0, 0] <= harm * (1 + 1e-12) and up[0, 0] >= harm * (1 - 1e-12)
    assert abs(up[1, 1] - arith) < 1e-10 * arith    # along the layers the minimiser is 0
    assert lo[1, 1] <= arith * (1 + 1e-12)


@pytest.mark.parametrize("seed,N", [(3, 9), (5, 15), (8, 11)])
def test_duality_and_ga_inside(seed, N):
    m = W.random_disk_instance(seed, N=N)
    mat = C.material_from_dict(m)
    up, lo, A, Binv, infos = GN.gani_bounds(mat, [N, N])
    assert all(i["converged"] for i in infos.values())
    scale = np.abs(A).max()
    assert np.abs(Binv - A).max() < 1e-9 * scale            # Remark duality_gani
    gup, glo, _ = G.bounds(mat, [N, N], tol=1e-12)
    # Loewner order lower_apost <= Ga lower <= Ga upper <= upper_apost
    for small, big in [(lo, glo), (glo, gup), (gup, up)]:
        assert np.linalg.eigvalsh(big - small).min() > -1e-10 * scale
