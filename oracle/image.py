"""Grid-based (pixel or voxel image) composites (FP64, CPU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

* image_table  -- Lemma grid_compos with psi the characteristic function of one
                  pixel (side h_a = 1/P_a, centred at the origin; the
                  piecewise-constant image of eq. gridcomp): the coefficient table
                      a^(m) = prod_a sinc(m_a / P_a) (1/|P|) sum_p C^p w_P^{-m.p},
                  m in Z_{2N-1}, evaluated with a P-sized DFT and read at
                  m mod P (Remark eval_with_FFT: truncated or periodically
                  enlarged).  Pixel p (array index p_a = 0 .. P_a - 1) is centred at
                  x = p / P (periodic).
* image_bounds -- the Ga bounds of the image: primal with the table of C, dual
                  with the table of 1/C (the inverse of a piecewise-constant
                  image is the piecewise-constant image of the inverses).
"""
from __future__ import annotations

import numpy as np

from . import galerkin as G
from .coefficients import _sinc, freq_grid
from .fourier import fdft_nd


def image_table(C: np.ndarray, N) -> np.ndarray:
    C = np.asarray(C, dtype=np.float64)
    P = C.shape
    d = len(P)
    Chat = fdft_nd(C.astype(np.complex128), axes=range(d))      # index = m mod P
    m = freq_grid([2 * n - 1 for n in N])
    val = Chat[tuple(np.mod(m[..., a], P[a]) for a in range(d))]
    for a in range(d):
        val = val * _sinc(m[..., a] / P[a])
    return val


def image_bounds(C: np.ndarray, N, M=None, tol: float = 1e-10):
    """(upper, lower): the Ga bounds of the piecewise-constant image C."""
    d = len(N)
    eye = np.eye(d)
    out = {}
    for kind, img in ((G.PRIMAL, C), (G.DUAL, 1.0 / np.asarray(C, dtype=np.float64))):
        op = G.Operator(None, N, kind, M=M, table=image_table(img, N))
        fields = [G.solve_load(op, eye[i], tol=tol)[0] for i in range(d)]
        out[kind] = G.gram(op, fields)
    lower = np.linalg.inv(out[G.DUAL])
    return out[G.PRIMAL], 0.5 * (lower + lower.T)
