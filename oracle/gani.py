"""GaNi scheme and its a-posteriori guaranteed bounds (FP64, CPU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

* sample_values -- the coefficient at the grid points x_N^k = k / N
                   (k_a = 0 .. N_a - 1), the data of the trapezoidal rule
                   (eq. approx_bilin).  Reading of the paper: it leaves points
                   on an inclusion's boundary open; here a point belongs to an
                   inclusion when its periodic distance to the centre is at most
                   the radius (DISK, SPHERE) or at most half the side along every
                   axis (BOX).
* GaNiOperator   -- Algorithm 1 on the Fourier side: inverse DFT of size N,
                   pointwise multiply by a(x_N^k), forward DFT (with 1/|N|),
                   projection.  It is ``galerkin.matvec_double_grid`` with the
                   double grid replaced by the N grid and A_M by the samples.
                   The bilinear form is the trapezoidal rule
                   (1/|N|) sum_k a(x^k) u(x^k).v(x^k) (eq. approx_bilin, with the
                   mean normalisation so that a constant coefficient gives a0).
* gani_bounds    -- Def. GaNi: minimisers e~_N, j~_N of the trapezoidal energies;
                   the GaNi matrices A~_N (primal) and B~_N (dual, returned
                   inverted); the a-posteriori matrices of eq. GaNi_apost, the
                   exact (Ga) energies of the GaNi minimisers, which are
                   guaranteed bounds (section "Structure of guaranteed bounds").
"""
from __future__ import annotations

import numpy as np

from . import galerkin as G
from .coefficients import BOX, Material, validate


def sample_values(mat: Material, N) -> np.ndarray:
    """a(x_N^k) on the grid x^k = k / N, shape N (C-order over k_a = 0..N_a-1)."""
    N = list(N)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) / n for n in N], indexing="ij")
    val = np.full(N, float(mat.a0))
    for inc in mat.inclusions:
        dist = []
        for a in range(len(N)):
            t = grids[a] - float(inc.center[a])
            dist.append(t - np.rint(t))                       # periodic offset in [-1/2, 1/2]
        if inc.shape == BOX:
            inside = np.ones(N, dtype=bool)
            for a in range(len(N)):
                inside &= np.abs(dist[a]) <= 0.5 * float(inc.size[a])
        else:
            r = float(inc.size[0])
            s = dist[0] * dist[0]
            for a in range(1, len(N)):
                s = s + dist[a] * dist[a]
            inside = s <= r * r
        val[inside] = float(inc.value)
    return val


class GaNiOperator:
    """G a~_N on Z_N (Algorithm 1): the trapezoidal-rule operator of the primal
    (coefficient a) or dual (coefficient 1/a) formulation."""

    def __init__(self, mat: Material, N, kind: str):
        validate(mat)
        self.N = list(N)
        self.d = len(N)
        self.kind = kind
        self.mat = mat if kind == G.PRIMAL else mat.inverse()
        self.a_N = sample_values(self.mat, self.N)

    def apply(self, x: np.ndarray, project_out: bool = True) -> np.ndarray:
        return G.matvec_double_grid(x, self.a_N, self.kind if project_out else None)

    def rhs(self, E) -> np.ndarray:
        """b = -G (a~ E)^: the load's image under the unprojected operator."""
        AE = self.apply(G.constant_field(E, self.N), project_out=False)
        return -G.project(AE, self.kind)

    def energy(self, v: np.ndarray, w: np.ndarray) -> float:
        """a~_N(v, w) = (1/|N|) sum_k a(x^k) v(x^k).w(x^k) by Parseval."""
        return G.inner(self.apply(v, project_out=False), w)


def gani_bounds(mat: Material, N, M=None, tol: float = 1e-12, maxiter: int = 10000):
    """Returns (upper, lower, A_gani, B_gani_inv, infos).

    upper = exact Gram a(v_i, v_j) of the d primal GaNi minimisers v_i = E_i + e~_i
    (eq. GaNi_apost), lower = inverse of the exact Gram a^{-1}(.,.) of the dual
    ones; A_gani = trapezoidal Gram of the primal minimisers (A~_N), B_gani_inv =
    inverse of the trapezoidal Gram of the dual ones (B~_N^{-1})."""
    d = len(N)
    eye = np.eye(d)
    exact = {}
    approx = {}
    infos = {}
    for kind in (G.PRIMAL, G.DUAL):
        opn = GaNiOperator(mat, N, kind)
        fields = []
        for i in range(d):
            b = opn.rhs(eye[i])
            e, info = G.cg(opn, b, tol, maxiter)
            fields.append(G.constant_field(eye[i], N) + G.admissible(e, kind))
            infos[(kind, i)] = info
        approx[kind] = G.gram(opn, fields)
        exact[kind] = G.gram(G.Operator(mat, N, kind, M=M), fields)
    sym = lambda X: 0.5 * (X + X.T)   # noqa: E731
    return (exact[G.PRIMAL], sym(np.linalg.inv(exact[G.DUAL])), approx[G.PRIMAL],
            sym(np.linalg.inv(approx[G.DUAL])), infos)
