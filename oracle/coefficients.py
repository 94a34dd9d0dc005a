"""Fourier coefficients of inclusion-matrix composites (FP64, CPU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

A scalar isotropic coefficient A(x) = a(x) I is described by a matrix value a0
and disjoint inclusions i = 1..n with shape f_i, centre x_i and inside value
a_i (eq. inclcomp with A_i = (a_i - a0) I):

    a(x) = a0 + sum_i (a_i - a0) f_i(x - x_i).

Its Fourier coefficients (Section 2.2: f^(k) = int_Y f(x) exp(-2 pi i k.x) dx)
are

    a^(n) = a0 delta_{n0} + sum_i (a_i - a0) exp(-2 pi i n.x_i) f_i^(n)     (*)

(the shift factor phi_{-n}(x_i) of eq. inclcomp_formula).  Because the
inclusions are disjoint, 1/a(x) = 1/a0 + sum_i (1/a_i - 1/a0) f_i(x - x_i) is of
the same form; its table is the dual coefficient table B^ used by the dual
problem (Cor. Ga_linsys, with B the coefficient of the inverse material).

Shape coefficients (Remark anal_Fourier, eq. char_func_Four):
  box  rect_h:  prod_a h_a sinc(h_a k_a),  sinc(x) = sin(pi x)/(pi x)
  disk circ_r:  pi r^2 at k = 0, else r J1(2 pi r |k|) / |k|
                (the paper's "r^2 B1(2 pi r|k|)/(r|k|)" with B1 = J1)
  ball (d = 3, not printed in the paper): 4 pi r^3 / 3 at k = 0, else
                (sin q - q cos q) / (2 pi^2 |k|^3),  q = 2 pi r |k|;
                for q < 1e-2 the Taylor series
                4 pi r^3/3 (1 - q^2/10 + q^4/280 - q^6/15120) avoids cancellation.
The ball formula follows from the radial Fourier transform in three dimensions,
F(rho) = 4 pi int_0^r s^2 sin(2 pi rho s)/(2 pi rho s) ds; the tests pin it to
that integral by quadrature.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import j1

from .fourier import centred_freqs

BOX, DISK, SPHERE = 0, 1, 2


@dataclass
class Inclusion:
    """One inclusion: shape (BOX/DISK/SPHERE), centre x_i, size, inside value a_i.

    ``size`` is the side vector h (BOX) or the radius r in size[0] (DISK/SPHERE).
    """
    shape: int
    center: tuple
    size: tuple
    value: float


@dataclass
class Material:
    """a(x) = a0 + sum_i (a_i - a0) f_i(x - x_i) on the unit cell (-1/2, 1/2)^d."""
    d: int
    a0: float
    inclusions: list = field(default_factory=list)

    def inverse(self) -> "Material":
        """The coefficient 1/a(x) of the same geometry (valid for disjoint inclusions)."""
        return Material(self.d, 1.0 / self.a0,
                        [Inclusion(i.shape, i.center, i.size, 1.0 / i.value) for i in self.inclusions])

    def volume_fractions(self):
        return [shape_coeff(i.shape, np.zeros((1, self.d)), i.size)[0].real for i in self.inclusions]

    def mean(self) -> float:
        """<a> = a^(0) (Section 2.2: the mean is the zero-frequency coefficient)."""
        return self.a0 + sum((i.value - self.a0) * f for i, f in zip(self.inclusions, self.volume_fractions()))

    def harmonic_mean(self) -> float:
        return 1.0 / self.inverse().mean()


def _sinc(x):
    """sin(pi x)/(pi x), 1 at 0 (the paper's sinc, Remark anal_Fourier).

    sin(pi x) is evaluated after reducing x modulo 2 (exact in binary floating
    point), so large arguments keep full relative accuracy."""
    x = np.asarray(x, dtype=np.float64)
    red = x - 2.0 * np.round(0.5 * x)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = np.sin(np.pi * red[nz]) / (np.pi * x[nz])
    return out


def shape_coeff(shape: int, k: np.ndarray, size) -> np.ndarray:
    """Fourier coefficient f^(k) of a centred characteristic function.

    ``k`` has shape (..., d) of integer frequencies.  Remark anal_Fourier.
    """
    k = np.asarray(k, dtype=np.float64)
    d = k.shape[-1]
    if shape == BOX:
        h = np.asarray(size, dtype=np.float64)[:d]
        out = np.ones(k.shape[:-1])
        for a in range(d):
            out = out * h[a] * _sinc(h[a] * k[..., a])
        return out.astype(np.complex128)
    r = float(size[0])
    rho = np.sqrt(np.sum(k * k, axis=-1))
    if shape == DISK:
        if d != 2:
            raise ValueError("disk inclusions are two-dimensional")
        out = np.empty(rho.shape)
        z = rho == 0
        out[z] = np.pi * r * r
        nz = ~z
        out[nz] = r * j1(2 * np.pi * r * rho[nz]) / rho[nz]
        return out.astype(np.complex128)
    if shape == SPHERE:
        if d != 3:
            raise ValueError("sphere inclusions are three-dimensional")
        q = 2 * np.pi * r * rho
        out = np.empty(rho.shape)
        small = q < 1e-2
        q2 = q[small] ** 2
        out[small] = 4.0 / 3.0 * np.pi * r ** 3 * (1 - q2 / 10 + q2 * q2 / 280 - q2 ** 3 / 15120)
        big = ~small
        qb = q[big]
        out[big] = (np.sin(qb) - qb * np.cos(qb)) / (2 * np.pi ** 2 * rho[big] ** 3)
        return out.astype(np.complex128)
    raise ValueError(f"unknown shape {shape}")


def coeff_at(mat: Material, n: np.ndarray) -> np.ndarray:
    """a^(n) of (*) at integer frequencies ``n`` of shape (..., d)."""
    n = np.asarray(n)
    out = np.zeros(n.shape[:-1], dtype=np.complex128)
    out[np.all(n == 0, axis=-1)] += mat.a0
    for inc in mat.inclusions:
        xi = np.asarray(inc.center, dtype=np.float64)[: mat.d]
        t = n.astype(np.float64) @ xi
        t = t - np.round(t)          # exp(-2 pi i t) is 1-periodic in t: reduce first
        phase = np.exp(-2j * np.pi * t)
        out += (inc.value - mat.a0) * phase * shape_coeff(inc.shape, n, inc.size)
    return out


def freq_grid(N) -> np.ndarray:
    """All k in Z_N (centred storage order) as an array of shape (*N, d)."""
    axes = [centred_freqs(n) for n in N]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


def coeff_table(mat: Material, N) -> np.ndarray:
    """a^(n) for n in Z_{2N-1}, centred (the table entering eq. MBA_GA)."""
    return coeff_at(mat, freq_grid([2 * n - 1 for n in N]))


def _overlap_at(a: Inclusion, b: Inclusion, delta: np.ndarray, d: int) -> bool:
    """Do the open interiors of inclusion a (centred at 0) and inclusion b
    (centred at delta) intersect?  Touching shapes do not overlap."""
    ra, rb = a.shape in (DISK, SPHERE), b.shape in (DISK, SPHERE)
    if ra and rb:                                    # two balls: centre distance
        return float(np.linalg.norm(delta)) < a.size[0] + b.size[0]
    if not ra and not rb:                            # two boxes: every axis overlaps
        return all(abs(delta[x]) < 0.5 * (a.size[x] + b.size[x]) for x in range(d))
    box, ball = (b, a) if ra else (a, b)
    off = delta if ra else -delta                    # ball centre relative to the box centre
    gap = np.maximum(np.abs(off) - 0.5 * np.asarray(box.size[:d], dtype=np.float64), 0.0)
    return float(np.linalg.norm(gap)) < ball.size[0]  # distance from the box to the ball centre


def validate(mat: Material) -> None:
    """Admissibility checks: SPD values (eq. A), inclusions that do not meet
    their own periodic images (box h_a <= 1, radius <= 1/2) and do not overlap
    each other or each other's periodic images (needed for the table of 1/a to
    be of the form (*)).  Every pair is checked against the 3^d nearest images
    of the second inclusion."""
    if not (mat.a0 > 0 and all(i.value > 0 for i in mat.inclusions)):
        raise ValueError("coefficients must be positive")
    for i in mat.inclusions:
        if i.shape == BOX and any(h <= 0 or h > 1 for h in i.size[: mat.d]):
            raise ValueError("box side must be in (0, 1]")
        if i.shape in (DISK, SPHERE) and not (0 < i.size[0] <= 0.5):
            raise ValueError("radius must be in (0, 1/2]")
    d = mat.d
    shifts = np.stack(np.meshgrid(*([np.arange(-1, 2)] * d), indexing="ij"), axis=-1).reshape(-1, d)
    incs = mat.inclusions
    for a in range(len(incs)):
        for b in range(a + 1, len(incs)):
            delta = (np.asarray(incs[b].center[:d], dtype=np.float64)
                     - np.asarray(incs[a].center[:d], dtype=np.float64))
            delta = delta - np.round(delta)
            for s in shifts:
                if _overlap_at(incs[a], incs[b], delta + s, d):
                    raise ValueError("inclusions overlap")


def material_from_dict(m: dict) -> Material:
    """Build a Material from the plain microstructure dict of ``workloads``."""
    incs = [Inclusion(int(s), tuple(c), tuple(z), float(v)) for (s, c, z, v) in m["inclusions"]]
    return Material(int(m["d"]), float(m["a0"]), incs)
