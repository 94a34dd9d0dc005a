"""Index sets and discrete Fourier transforms of the oracle (FP64, CPU).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Conventions (Section 4.1 and Section 5.1 of the paper):

* Z_N = {k in Z^d : -N_a/2 <= k_a < N_a/2} (eq. index_set).  For odd N this is
  the symmetric set {-(N-1)/2 .. (N-1)/2}; arrays on Z_N are stored *centred*:
  array index i holds frequency k = i - (N-1)//2.  For even M the set Z_M holds
  -M/2 .. M/2-1; on a double grid we store values *wrapped*: index m holds the
  grid point x_M^m = m/M (m and m-M denote the same point of the periodic cell).
* DFT coefficients omega_M^{kn} = exp(2 pi i sum_a k_a n_a / M_a)
  (eq. DFT_coef).  The inverse DFT (F^{-1} in eq. DFT) is unscaled and carries
  the + sign; the forward DFT carries the - sign and the factor 1/|M|.

The FFT here is the oracle's own: a recursive decimation-in-time split on the
smallest prime factor, a naive O(L^2) DFT for small prime lengths and
Bluestein's chirp-z identity (k n = (k^2 + n^2 - (k-n)^2)/2) for large prime
lengths.  It is pinned against the naive DFT and numpy.fft in the tests.
"""
from __future__ import annotations

import numpy as np

_NAIVE_PRIME_MAX = 64


def centred_freqs(n: int) -> np.ndarray:
    """Frequencies of Z_n in storage order (eq. index_set, Def. trig_pol).

    For odd n: -(n-1)/2 .. (n-1)/2.  For even n: -n/2 .. n/2-1.
    """
    return np.arange(n) - n // 2


def wrapped_freqs(m: int) -> np.ndarray:
    """Frequency (in Z_m) held at wrapped storage index j = 0..m-1."""
    j = np.arange(m)
    return np.where(j < (m + 1) // 2, j, j - m) if m % 2 else np.where(j < m // 2, j, j - m)


def smallest_prime_factor(n: int) -> int:
    if n % 2 == 0:
        return 2
    p = 3
    while p * p <= n:
        if n % p == 0:
            return p
        p += 2
    return n


def _root(sign: int, num: np.ndarray, den: int) -> np.ndarray:
    """exp(sign * 2 pi i * num/den) with num reduced mod den first (accuracy)."""
    r = np.mod(num, den).astype(np.float64) / den
    return np.exp(sign * 2j * np.pi * r)


def naive_dft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """X[k] = sum_n x[n] exp(sign 2 pi i k n / L) along the last axis (definition)."""
    L = x.shape[-1]
    n = np.arange(L)
    D = _root(sign, np.outer(n, n), L)
    return x @ D.T


def _bluestein_last(x: np.ndarray, sign: int) -> np.ndarray:
    """Prime-length DFT by the chirp-z identity, convolution by a power-of-two FFT."""
    L = x.shape[-1]
    n = np.arange(L)
    chirp = np.exp(sign * 1j * np.pi * (np.mod(n * n, 2 * L).astype(np.float64) / L))
    P = 1
    while P < 2 * L - 1:
        P *= 2
    a = np.zeros(x.shape[:-1] + (P,), dtype=np.complex128)
    a[..., :L] = x * chirp
    b = np.zeros(P, dtype=np.complex128)
    b[:L] = np.conj(chirp)
    b[P - L + 1:] = np.conj(chirp[1:])[::-1]
    A = _fft_last(a, -1)
    B = _fft_last(b, -1)
    conv = _fft_last(A * B, +1) / P
    return chirp * conv[..., :L]


def _fft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """Unscaled DFT with exponent sign ``sign`` along the last axis (recursive)."""
    x = np.asarray(x, dtype=np.complex128)
    L = x.shape[-1]
    if L == 1:
        return x.copy()
    p = smallest_prime_factor(L)
    if p == L:
        if L <= _NAIVE_PRIME_MAX:
            return naive_dft_last(x, sign)
        return _bluestein_last(x, sign)
    m = L // p
    # decimation in time: subsequence q holds x[q + p*n], n = 0..m-1
    sub = np.moveaxis(x.reshape(x.shape[:-1] + (m, p)), -1, 0)
    Y = _fft_last(sub, sign)                                   # (p, ..., m)
    q = np.arange(p).reshape((p,) + (1,) * (Y.ndim - 1))
    k = np.arange(m)
    Z = Y * _root(sign, q * k, L)                              # twiddles w_L^{qk}
    D = _root(sign, np.outer(np.arange(p), np.arange(p)), p)   # w_p^{jq}
    W = np.tensordot(D, Z, axes=([1], [0]))                    # (p_j, ..., m)
    # X[k + m j] = W[j, ..., k]
    W = np.moveaxis(W, 0, -2)                                  # (..., p, m)
    return W.reshape(W.shape[:-2] + (L,))


def dft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    """Unscaled DFT along ``axis`` with exponent sign ``sign`` (+1 inverse, -1 forward)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(x, sign), -1, axis)


def idft_nd(x: np.ndarray, axes) -> np.ndarray:
    """F^{-1}: u[m] = sum_k x[k] omega^{mk} over ``axes`` (unscaled, eq. DFT)."""
    for ax in axes:
        x = dft_axis(x, ax, +1)
    return x


def fdft_nd(x: np.ndarray, axes) -> np.ndarray:
    """F: X[k] = (1/|M|) sum_m x[m] omega^{-mk} over ``axes`` (eq. DFT)."""
    size = 1
    for ax in axes:
        x = dft_axis(x, ax, -1)
        size *= x.shape[ax]
    return x / size


def pad_centred_to_wrapped(xc: np.ndarray, M, lead: int = 0) -> np.ndarray:
    """Place coefficients stored centred on Z_N into a zero array of shape M at
    wrapped positions k mod M (the zero padding of Algorithm 2 / eq. trig_conn_raw).

    ``lead`` leading axes (e.g. the vector component) are kept as they are.
    """
    shp = xc.shape[lead:]
    out = np.zeros(xc.shape[:lead] + tuple(M), dtype=np.complex128)
    idx = tuple(np.mod(centred_freqs(n), m) for n, m in zip(shp, M))
    out[(Ellipsis,) + np.ix_(*idx)] = xc
    return out


def truncate_wrapped_to_centred(xw: np.ndarray, N, lead: int = 0) -> np.ndarray:
    """Gather the entries k in Z_N (stored wrapped on Z_M) into a centred array."""
    M = xw.shape[lead:]
    idx = tuple(np.mod(centred_freqs(n), m) for n, m in zip(N, M))
    return xw[(Ellipsis,) + np.ix_(*idx)]
