"""Seeded synthetic inputs (microstructures and request streams).

This module draws inclusion geometries, contrasts and grid orders only; it holds
none of the method's arithmetic (no Fourier coefficients, no transforms, no
solver).  It is the one module shared by the CPU oracle tests and the GPU path.

A microstructure is a plain dict:
    {"d": 2 or 3, "N": [odd ints], "a0": matrix value,
     "inclusions": [(shape, center(tuple of 3), size(tuple of 3), inside value), ...]}
with shape 0 = box (size = side lengths), 1 = disk (d = 2, size[0] = radius),
2 = sphere (d = 3, size[0] = radius).  The unit cell is (-1/2, 1/2)^d.

The recipes follow the paper's Section 7 problems (square and circular
inclusions of contrast 10..1e4 in a unit cell) at the sizes of the workloads
this library is measured on; the base seed is 20141206 and instance i of a batch
uses seed + i (NumPy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20141206
BOX, DISK, SPHERE = 0, 1, 2


def _micro(d, N, a0, incs):
    return {"d": d, "N": [int(n) for n in N], "a0": float(a0), "inclusions": incs}


def centred_square(N=15, side=1 / math.sqrt(2), value=10.0):
    """d = 2, centred square of side 1/sqrt(2) (volume fraction 0.5), a = 1 | 10."""
    return _micro(2, [N, N], 1.0, [(BOX, (0.0, 0.0, 0.0), (side, side, 1.0), value)])


def centred_disk(N, fraction=0.3, value=100.0):
    """d = 2, one centred disk of volume fraction 0.3 (r = sqrt(0.3/pi)), contrast 100."""
    r = math.sqrt(fraction / math.pi)
    return _micro(2, [N, N], 1.0, [(DISK, (0.0, 0.0, 0.0), (r, 0.0, 0.0), value)])


def centred_sphere(N, fraction=0.2, value=1000.0):
    """d = 3, one centred sphere of volume fraction 0.2 (r = (3 f / 4 pi)^(1/3)), contrast 1000."""
    r = (3 * fraction / (4 * math.pi)) ** (1 / 3)
    return _micro(3, [N, N, N], 1.0, [(SPHERE, (0.0, 0.0, 0.0), (r, 0.0, 0.0), value)])


def centred_cube(N, side=0.6, value=1000.0):
    """d = 3, one centred cube of side 0.6 (volume fraction 0.216), contrast 1000."""
    return _micro(3, [N, N, N], 1.0, [(BOX, (0.0, 0.0, 0.0), (side, side, side), value)])


def laminate(N, d=2, h=0.4, value=5.0, a0=1.0, center=0.1):
    """A box spanning the cell in every direction but the first: layers normal to e_1."""
    size = (h, 1.0, 1.0)
    return _micro(d, [N] * d, a0, [(BOX, (center, 0.0, 0.0), size, value)])


def _torus_dist(a, b):
    delta = np.asarray(a) - np.asarray(b)
    delta = delta - np.round(delta)
    return float(np.linalg.norm(delta))


def random_balls(rng, d, count, rmin, rmax, max_tries=10000):
    """Non-overlapping disks (d = 2) or spheres (d = 3) with radius U(rmin, rmax)
    and centres U[-1/2, 1/2)^d, rejection-sampled in the torus distance."""
    placed = []
    tries = 0
    while len(placed) < count and tries < max_tries:
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(-0.5, 0.5, size=d)
        if all(_torus_dist(c, pc) > r + pr for pc, pr in placed):
            placed.append((c, r))
    return placed


def random_disk_instance(seed, N=None):
    """One instance of the 512-instance batch: K ~ U{1..20} disks, r ~ U(0.03, 0.12),
    contrast log-uniform in [2, 1e4], N uniform over odd 31..255."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 21))
    contrast = float(np.exp(rng.uniform(math.log(2.0), math.log(1e4))))
    if N is None:
        N = int(2 * rng.integers(15, 128) + 1)          # odd 31..255
    balls = random_balls(rng, 2, K, 0.03, 0.12)
    incs = [(DISK, (float(c[0]), float(c[1]), 0.0), (float(r), 0.0, 0.0), contrast) for c, r in balls]
    return _micro(2, [N, N], 1.0, incs)


def disk_batch(count=512, seed=BASE_SEED, N=None):
    """The batched workload: ``count`` seeded disk instances (instance i uses seed + i)."""
    return [random_disk_instance(seed + i, N=N) for i in range(count)]


def random_sphere_instance(seed, N=None):
    """d = 3 served request: 1..8 non-overlapping spheres r ~ U(0.05, 0.2),
    contrast log-uniform in [2, 1e3], N odd uniform in 15..129."""
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 9))
    contrast = float(np.exp(rng.uniform(math.log(2.0), math.log(1e3))))
    if N is None:
        N = int(2 * rng.integers(7, 65) + 1)            # odd 15..129
    balls = random_balls(rng, 3, K, 0.05, 0.2)
    incs = [(SPHERE, tuple(float(v) for v in c), (float(r), 0.0, 0.0), contrast) for c, r in balls]
    return _micro(3, [N, N, N], 1.0, incs)


def voxel_foam(P=99, seed=BASE_SEED + 7, porosity=0.6, count=60):
    """A seeded two-phase voxel image of size P^3 standing in for the fly-ash
    foam image (Section 7.5, not available): pores are random overlapping balls
    (radius U(0.05, 0.15), centres uniform) until the pore fraction reaches
    `porosity`; solid voxels carry 0.49 and pore voxels 0.029 (the foam's phase
    values).  Voxel p is centred at p / P (periodic)."""
    rng = np.random.default_rng(seed)
    x = np.arange(P) / P
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    pore = np.zeros((P, P, P), dtype=bool)
    for _ in range(count * 10):
        if pore.mean() >= porosity:
            break
        c = rng.uniform(0.0, 1.0, 3)
        r = rng.uniform(0.05, 0.15)
        d2 = np.zeros_like(X)
        for g, cc in zip((X, Y, Z), c):
            t = g - cc
            t = t - np.rint(t)
            d2 = d2 + t * t
        pore |= d2 <= r * r
    return np.where(pore, 0.029, 0.49)


def request_stream(rate=200.0, duration=60.0, seed=BASE_SEED, d3_share=0.5,
                   n2=(63, 1023), n3=(15, 129)):
    """Poisson arrivals (mean ``rate`` per second) of bound requests mixing
    d = 2 disk instances (N odd in n2) and d = 3 sphere instances (N odd in n3).
    Returns a list of (arrival_time_s, microstructure)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            break
        s = seed + 1000 + i
        if rng.uniform() < d3_share:
            N = int(2 * rng.integers((n3[0] - 1) // 2, (n3[1] - 1) // 2 + 1) + 1)
            m = random_sphere_instance(s, N=N)
        else:
            N = int(2 * rng.integers((n2[0] - 1) // 2, (n2[1] - 1) // 2 + 1) + 1)
            m = random_disk_instance(s, N=N)
        out.append((t, m))
        i += 1
    return out


def random_field(rng, d, N, hermitian=True):
    """A random trial field on Z_N (d components, centred storage), Hermitian
    (x(-k) = conj x(k)) so that it is a real trigonometric polynomial."""
    shape = (d,) + tuple(N)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if hermitian:
        flip = x[(slice(None),) + (slice(None, None, -1),) * d]
        x = 0.5 * (x + np.conj(flip))
    return x
