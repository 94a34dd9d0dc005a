"""Ga scheme: projections, Galerkin operator, conjugate gradients, bounds (FP64, CPU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Fields are trigonometric polynomials of odd order N (Def. trig_pol) stored by
their Fourier coefficients on Z_N, centred, as complex arrays of shape
(d, N_1, ..., N_d) (the vector component first).  The material is isotropic,
A(x) = a(x) I, with coefficient table a^(n), n in Z_{2N-1}
(``coefficients.coeff_table``).

Operators written out (each is the plain definition from the cited passage):

* projection(k) -- Def. projection:  G_E(k) = k (x) k / k.k,  G_J(k) = I - G_E(k),
                   both zero at k = 0.
* dense_galerkin -- Lemma FD_matrix_full:  (A^full)^{lk} = a^(l - k), l, k in Z_N.
* double_grid_values -- eq. MBA_GA:  A_M(x_m) = sum_{n in Z_{2N-1}} omega_M^{mn} a^(n).
* matvec_double_grid -- Algorithm 2 written on the Fourier side (Cor.
                   Ga_linsys, item 1 composed with the DFT): zero-pad Z_N -> Z_M,
                   inverse DFT, multiply by A_M, forward DFT (with 1/|M|),
                   truncate to Z_N, project.  By Lemma integ_eval_VM this equals
                   G A^full for every M >= 2N-1.
* reduced_matvec -- the same operator by Lemma reduce_grid (Algorithm 3): 2^d
                   shifted N-size transforms with the double-grid values of
                   M = 2N read at the points 2r - s.
* matvec_sampled -- the same operator at chosen output frequencies, directly
                   from the definition y(l) = G(l) sum_k a^(l-k) x(k)
                   (O(|N|) per output; usable at any N).
* prolong        -- the coarse-to-fine prolongation of Section 7.4 (zero
                   coefficients at the new frequencies: the same polynomial).
* cg             -- conjugate gradients (Remark CG; Saad's Algorithm 6.18) on
                   the range of the projection, x0 = 0, stop when
                   ||r_k||_2 / ||b||_2 <= tol (the 2-norm over Z_N coefficients,
                   equal to the L2 norm by Parseval).
* bounds         -- upper U_ij = a(E_i + e_i, E_j + e_j) (eq. GA_prim) and lower
                   L = D^{-1} with D_ij = a^{-1}(J_i + j_i, J_j + j_j)
                   (Prop. struct_bounds, eq. spd_inverse_ineq), symmetrised.
"""
from __future__ import annotations

import math

import numpy as np

from .coefficients import Material, coeff_at, coeff_table, freq_grid, validate
from .fourier import (centred_freqs, fdft_nd, idft_nd, pad_centred_to_wrapped,
                      truncate_wrapped_to_centred)

PRIMAL, DUAL = "primal", "dual"


# ----------------------------------------------------------------------------
# projections (Def. projection, Def. discrete_proj)
# ----------------------------------------------------------------------------
def projection_matrices(N, kind: str) -> np.ndarray:
    """G(k) for all k in Z_N, shape (*N, d, d).  kind: PRIMAL -> G_E, DUAL -> G_J."""
    k = freq_grid(N).astype(np.float64)
    d = len(N)
    kk = np.einsum("...a,...b->...ab", k, k)
    n2 = np.sum(k * k, axis=-1)
    zero = n2 == 0
    n2 = np.where(zero, 1.0, n2)
    GE = kk / n2[..., None, None]
    GE[zero] = 0.0
    if kind == PRIMAL:
        return GE
    GJ = np.eye(d) - GE
    GJ[zero] = 0.0
    return GJ


def project(x: np.ndarray, kind: str) -> np.ndarray:
    """y(k) = G(k) x(k) for a field x of shape (d, *N)."""
    N = x.shape[1:]
    G = projection_matrices(N, kind)
    return np.einsum("...ab,b...->a...", G, x)


# ----------------------------------------------------------------------------
# the Galerkin operator
# ----------------------------------------------------------------------------
def default_M(N):
    """The smallest admissible double grid, M = 2N - 1 (Lemma integ_eval_VM)."""
    return [2 * n - 1 for n in N]


def double_grid_values(table: np.ndarray, M) -> np.ndarray:
    """A_M(x_m) = sum_{n in Z_{2N-1}} omega_M^{mn} a^(n) on the wrapped grid
    m = 0..M-1 (eq. MBA_GA).  Real up to rounding; the real part is returned."""
    NN = table.shape
    if any(m < nn for m, nn in zip(M, NN)):
        raise ValueError("M must be >= 2N - 1")
    padded = pad_centred_to_wrapped(table, M)
    vals = idft_nd(padded, axes=range(len(M)))
    return vals.real


def matvec_double_grid(x: np.ndarray, a_M: np.ndarray, kind: str) -> np.ndarray:
    """G A^full x through the double grid (Algorithm 2 on the Fourier side)."""
    d = x.shape[0]
    N = x.shape[1:]
    M = a_M.shape
    axes = range(1, d + 1)
    u = idft_nd(pad_centred_to_wrapped(x, M, lead=1), axes)      # values on the M-grid
    w = u * a_M[None]                                             # pointwise A_M
    wh = fdft_nd(w, axes)                                         # forward DFT, 1/|M|
    y = truncate_wrapped_to_centred(wh, N, lead=1)                # keep Z_N
    return project(y, kind) if kind is not None else y


def reduced_matvec(x: np.ndarray, a_2N: np.ndarray, kind) -> np.ndarray:
    """G A^full x by Lemma reduce_grid (Algorithm 3), for the double grid 2N:
    A^full = 2^-d sum_{s in {0,1}^d} S*(s) F_N A_N(s) F_N^{-1} S(s) with
    S(s) = diag(omega_{2N}^{-s.m}), m in Z_N, and A_N(s) the values of the 2N grid
    at the points 2r - s, r in Z_N (wrapped: the values at x = r/N - s/(2N))."""
    d = x.shape[0]
    N = list(x.shape[1:])
    axes = range(1, d + 1)
    m = [centred_freqs(n) for n in N]
    y = np.zeros_like(x, dtype=np.complex128)
    for s in np.ndindex(*([2] * d)):
        ph = np.ones(N, dtype=np.complex128)
        for a in range(d):
            shape = [1] * d
            shape[a] = N[a]
            ph = ph * np.exp(-1j * np.pi * s[a] * m[a] / N[a]).reshape(shape)   # omega_{2N}^{-s m}
        u = idft_nd(pad_centred_to_wrapped(x * ph[None], N, lead=1), axes)       # values at r/N - s/(2N)
        idx = np.ix_(*[(2 * np.arange(n) - sa) % (2 * n) for n, sa in zip(N, s)])
        w = u * a_2N[idx][None]
        wh = truncate_wrapped_to_centred(fdft_nd(w, axes), N, lead=1)
        y = y + np.conj(ph)[None] * wh
    y = y / 2 ** d
    return project(y, kind) if kind is not None else y


def dense_galerkin(table: np.ndarray, N) -> np.ndarray:
    """Scalar fully populated matrix (A^full)^{lk} = a^(l-k), shape (|N|, |N|)
    in C-order over centred Z_N (Lemma FD_matrix_full)."""
    k = freq_grid(N).reshape(-1, len(N))
    diff = k[:, None, :] - k[None, :, :]                    # l - k
    c = [(nn - 1) // 2 for nn in table.shape]               # centre of Z_{2N-1}
    idx = tuple(diff[..., a] + c[a] for a in range(len(N)))
    return table[idx]


def matvec_dense(x: np.ndarray, table: np.ndarray, kind) -> np.ndarray:
    """G A^full x with the dense matrix (brute force for tiny N)."""
    d = x.shape[0]
    N = x.shape[1:]
    A = dense_galerkin(table, N)
    y = (x.reshape(d, -1) @ A.T).reshape(x.shape)
    return project(y, kind) if kind is not None else y


def matvec_sampled(x: np.ndarray, mat: Material, kind, out_idx: np.ndarray) -> np.ndarray:
    """y(l) = G(l) sum_{k in Z_N} a^(l - k) x(k) at the output frequencies
    ``out_idx`` (shape (s, d), integer frequencies in Z_N).  Returns (s, d)."""
    d = x.shape[0]
    N = x.shape[1:]
    k = freq_grid(N).reshape(-1, d)
    xs = x.reshape(d, -1)
    out = np.empty((len(out_idx), d), dtype=np.complex128)
    for s, l in enumerate(np.asarray(out_idx)):
        a = coeff_at(mat, l[None, :] - k)                  # a^(l - k) for all k
        v = xs @ a                                         # (d,)
        out[s] = v
        if kind is not None:
            lf = l.astype(np.float64)
            n2 = lf @ lf
            GE = np.zeros((d, d)) if n2 == 0 else np.outer(lf, lf) / n2
            G = GE if kind == PRIMAL else (np.zeros((d, d)) if n2 == 0 else np.eye(d) - GE)
            out[s] = G @ v
    return out


# ----------------------------------------------------------------------------
# right-hand side, energies, CG
# ----------------------------------------------------------------------------
def inner(x: np.ndarray, y: np.ndarray) -> float:
    """Re sum_k x(k) . conj(y(k)) (the scalar product on C^{d x N}, Section 5.1)."""
    return float(np.real(np.vdot(y, x)))


def inner_exact(x: np.ndarray, y: np.ndarray) -> float:
    """The same scalar product with the sum of the products Re x conj y =
    x_re y_re + x_im y_im correctly rounded (math.fsum), so that the only
    rounding left in an energy is that of its operands.  Used for the bound
    energies (eq. GA_prim), whose terms cancel at high contrast."""
    xr, xi = np.real(x).ravel(), np.imag(x).ravel()
    yr, yi = np.real(y).ravel(), np.imag(y).ravel()
    return math.fsum(np.concatenate((xr * yr, xi * yi)))


def constant_field(E, N) -> np.ndarray:
    """The constant field E as coefficients on Z_N: E at k = 0, zero elsewhere."""
    d = len(N)
    f = np.zeros((d,) + tuple(N), dtype=np.complex128)
    f[(slice(None),) + tuple((n - 1) // 2 for n in N)] = np.asarray(E, dtype=np.float64)
    return f


def prolong(x: np.ndarray, N) -> np.ndarray:
    """I_N o I_M^{-1} (Section 7.4): the coefficients on Z_N of the trigonometric
    polynomial with coefficients x on a smaller odd grid, zero elsewhere."""
    d = x.shape[0]
    Nc = x.shape[1:]
    out = np.zeros((d,) + tuple(N), dtype=np.complex128)
    sl = tuple(slice((n - nc) // 2, (n - nc) // 2 + nc) for n, nc in zip(N, Nc))
    out[(slice(None),) + sl] = x
    return out


def rhs(table: np.ndarray, N, E, kind: str) -> np.ndarray:
    """b = -G A^full E^ (Prop. min2linear_sys); (A^full E^)(l) = a^(l) E."""
    d = len(N)
    c = [(nn - 1) // 2 for nn in table.shape]
    sl = tuple(slice(ci - (n - 1) // 2, ci + (n - 1) // 2 + 1) for ci, n in zip(c, N))
    a_N = table[sl]                                          # a^(l), l in Z_N
    AE = np.asarray(E, dtype=np.float64).reshape((d,) + (1,) * d) * a_N[None]
    return -project(AE, kind)


class Operator:
    """G A^full on Z_N for one material (primal) or its inverse (dual)."""

    def __init__(self, mat: Material, N, kind: str, M=None, method: str = "double_grid", table=None):
        """``table``: the coefficient table on Z_{2N-1} of this kind's coefficient
        when the material is not an inclusion-matrix composite (then ``mat`` may
        be None), e.g. ``image.image_table`` of a pixel image."""
        self.N = list(N)
        self.d = len(N)
        self.kind = kind
        if table is None:
            validate(mat)
            self.mat = mat if kind == PRIMAL else mat.inverse()
            self.table = coeff_table(self.mat, self.N)
        else:
            self.mat = None
            self.table = np.asarray(table, dtype=np.complex128)
        self.M = list(M) if M is not None else default_M(self.N)
        self.method = method
        if method == "double_grid":
            self.a_M = double_grid_values(self.table, self.M)
        elif method == "dense":
            self.A = dense_galerkin(self.table, self.N)
        else:
            raise ValueError(method)

    def apply(self, x: np.ndarray, project_out: bool = True) -> np.ndarray:
        kind = self.kind if project_out else None
        if self.method == "double_grid":
            return matvec_double_grid(x, self.a_M, kind)
        d = self.d
        y = (x.reshape(d, -1) @ self.A.T).reshape(x.shape)
        return project(y, kind) if kind is not None else y

    def rhs(self, E) -> np.ndarray:
        return rhs(self.table, self.N, E, self.kind)

    def energy(self, v: np.ndarray, w: np.ndarray) -> float:
        """a(v, w) = Re sum_l conj(w(l)) . (A^full v)(l) (Lemma FD_matrix_full)."""
        return inner_exact(self.apply(v, project_out=False), w)


def cg(op: Operator, b: np.ndarray, tol: float, maxiter: int = 10000, x0=None, track_energy_E=None):
    """Conjugate gradients on the range of G (Remark CG), x0 = 0 unless given.

    Returns (x, info) with info = {iters, relres, converged, energies}.  When
    ``track_energy_E`` is given, the energy a(E + x_k, E + x_k) after each
    iterate is recorded (the bound during CG, Section 7.4).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - op.apply(x) if x0 is not None else b.copy()
    bn = np.sqrt(inner(b, b))
    energies = []
    E_field = None
    if track_energy_E is not None:
        E_field = constant_field(track_energy_E, op.N)
        energies.append(op.energy(E_field + x, E_field + x))
    if bn == 0.0:
        return x, dict(iters=0, relres=0.0, converged=True, energies=energies)
    p = r.copy()
    rr = inner(r, r)
    it = 0
    relres = np.sqrt(rr) / bn
    while relres > tol and it < maxiter:
        q = op.apply(p)
        pq = inner(p, q)
        if not pq > 0:
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = inner(r, r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
        relres = np.sqrt(rr) / bn
        if E_field is not None:
            energies.append(op.energy(E_field + x, E_field + x))
    return x, dict(iters=it, relres=relres, converged=relres <= tol, energies=energies)


def solve_dense(op: Operator, b: np.ndarray) -> np.ndarray:
    """Direct solve of G A^full e = b on range(G) via the SPD system
    (G A G + (I - G)) e = b (for tiny N)."""
    d, N = op.d, op.N
    n = int(np.prod(N))
    A = op.A if op.method == "dense" else dense_galerkin(op.table, N)
    G = projection_matrices(N, op.kind).reshape(n, d, d)
    # big matrices indexed [(a, k), (b, l)]
    Gb = np.zeros((d, n, d, n))
    for a in range(d):
        for c in range(d):
            Gb[a, :, c, :] = np.diag(G[:, a, c])
    Gb = Gb.reshape(d * n, d * n)
    Ab = np.kron(np.eye(d), A)
    K = Gb @ Ab @ Gb + (np.eye(d * n) - Gb)
    e = np.linalg.solve(K, b.reshape(-1))
    return e.reshape(b.shape)


def gram(op: Operator, fields) -> np.ndarray:
    """Symmetrised Gram matrix X_ij = a(v_i, v_j) of the admissible fields v_i."""
    m = len(fields)
    Av = [op.apply(v, project_out=False) for v in fields]
    X = np.array([[inner_exact(Av[i], fields[j]) for j in range(m)] for i in range(m)])
    return 0.5 * (X + X.T)


def admissible(e: np.ndarray, kind: str) -> np.ndarray:
    """The nearest admissible fluctuation: the Hermitian part (the coefficients
    of a real trigonometric polynomial, Def. trig_pol: e(-k) = conj e(k)),
    projected onto the range of G (Def. projection).  Exact on admissible
    fields; applied to a computed minimiser it removes the rounding left outside
    E_N (J_N), so that its energy is that of an admissible field (Def. Ga)."""
    d = e.shape[0]
    flip = e[(slice(None),) + (slice(None, None, -1),) * d]
    return project(0.5 * (e + np.conj(flip)), kind)


def solve_load(op: Operator, E, tol: float = 1e-10, method: str = "cg", maxiter: int = 10000):
    """Minimiser e of a(E + e, E + e) over E_N (primal) or J_N (dual) and the
    admissible field v = E + e, with e made exactly admissible (``admissible``).
    Returns (v, info)."""
    b = op.rhs(E)
    if method == "cg":
        e, info = cg(op, b, tol, maxiter)
    else:
        e, info = solve_dense(op, b), dict(iters=0, relres=0.0, converged=True, energies=[])
    return constant_field(E, op.N) + admissible(e, op.kind), info


def _solve_task(args):
    """One load of ``bounds`` (module level so that a process pool can run it)."""
    mat, N, kind, M, op_method, E, tol, method, maxiter = args
    op = Operator(mat, N, kind, M=M, method=op_method)
    return solve_load(op, E, tol=tol, method=method, maxiter=maxiter)


def bounds(mat: Material, N, M=None, tol: float = 1e-10, method: str = "cg",
           op_method: str = "double_grid", maxiter: int = 10000, pool=None):
    """Guaranteed bounds of the Ga scheme (Def. Ga, Prop. struct_bounds).

    Returns (upper, lower, infos): upper = Gram of the d primal admissible
    fields in a(.,.), lower = inverse of the Gram of the d dual fields in
    a^{-1}(.,.) (eq. spd_inverse_ineq).  The 2d solves are independent; with
    ``pool`` (an executor with ``map``) they run there, else one after another.
    """
    d = len(N)
    eye = np.eye(d)
    tasks = [(mat, list(N), kind, M, op_method, eye[i], tol, method, maxiter)
             for kind in (PRIMAL, DUAL) for i in range(d)]
    solved = list(pool.map(_solve_task, tasks)) if pool is not None else [_solve_task(t) for t in tasks]
    out = {}
    infos = {}
    for kind in (PRIMAL, DUAL):
        op = Operator(mat, N, kind, M=M, method=op_method)
        fields = []
        for i in range(d):
            v, info = solved[(0 if kind == PRIMAL else d) + i]
            fields.append(v)
            infos[(kind, i)] = info
        out[kind] = gram(op, fields)
    upper = out[PRIMAL]
    lower = np.linalg.inv(out[DUAL])
    lower = 0.5 * (lower + lower.T)
    return upper, lower, infos
