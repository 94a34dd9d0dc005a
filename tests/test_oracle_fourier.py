"""Pins of the oracle's DFT/FFT (Section 4.1 eq. DFT_coef, Section 5.1 eq. DFT).

The oracle FFT is checked against (a) the DFT definition summed directly,
(b) numpy.fft (an independent library routine the oracle does not call),
(c) Parseval and inversion identities, and (d) the evaluation of a
trigonometric polynomial at grid points (eq. trig_conn_raw).
"""
import numpy as np
import pytest

from oracle import fourier as F

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 9, 12, 15, 29, 30, 49, 67, 97, 128, 135, 162, 270, 486]


@pytest.mark.parametrize("L", LENGTHS)
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_direct_sum(L, sign):
    rng = np.random.default_rng(L)
    x = rng.standard_normal((2, L)) + 1j * rng.standard_normal((2, L))
    n = np.arange(L)
    # direct sum of the definition, element by element (no matrix helper)
    ref = np.array([[sum(x[b, j] * np.exp(sign * 2j * np.pi * k * j / L) for j in n) for k in n]
                    for b in range(2)])
    got = F.dft_axis(x, 1, sign)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("L", LENGTHS + [4373 // 11, 211, 1024, 4374])
def test_fft_matches_numpy(L):
    rng = np.random.default_rng(1000 + L)
    x = rng.standard_normal((3, L)) + 1j * rng.standard_normal((3, L))
    assert np.allclose(F.dft_axis(x, 1, -1), np.fft.fft(x, axis=1), rtol=0, atol=1e-11 * np.sqrt(L))
    assert np.allclose(F.dft_axis(x, 1, +1), L * np.fft.ifft(x, axis=1), rtol=0, atol=1e-11 * np.sqrt(L))


def test_nd_roundtrip_and_parseval():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((6, 10, 15)) + 1j * rng.standard_normal((6, 10, 15))
    X = F.fdft_nd(x, axes=range(3))
    assert np.allclose(F.idft_nd(X, axes=range(3)), x, atol=1e-13)
    # Parseval for the scaled forward transform: sum|x|^2 = |M| sum|X|^2
    assert np.isclose(np.sum(np.abs(x) ** 2), x.size * np.sum(np.abs(X) ** 2), rtol=1e-13)


@pytest.mark.parametrize("N,M", [(5, 9), (5, 12), (7, 13), (7, 16)])
def test_idft_of_padded_coefficients_is_polynomial_value(N, M):
    """eq. trig_conn_raw: the inverse DFT of zero-padded coefficients equals the
    trigonometric polynomial evaluated at the grid points x_M^m = m/M."""
    rng = np.random.default_rng(N * M)
    c = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    vals = F.idft_nd(F.pad_centred_to_wrapped(c, [M, M]), axes=range(2))
    k = F.centred_freqs(N)
    for m in [(0, 0), (1, 3), (M - 1, 2), (M // 2, M - 1)]:
        x = np.array(m) / M
        direct = sum(c[i, j] * np.exp(2j * np.pi * (k[i] * x[0] + k[j] * x[1]))
                     for i in range(N) for j in range(N))
        assert abs(vals[m] - direct) < 1e-12 * np.abs(c).sum()


def test_index_sets():
    assert list(F.centred_freqs(5)) == [-2, -1, 0, 1, 2]
    assert list(F.centred_freqs(4)) == [-2, -1, 0, 1]         # Z_M for even M holds -M/2
    assert list(F.wrapped_freqs(5)) == [0, 1, 2, -2, -1]
    assert list(F.wrapped_freqs(6)) == [0, 1, 2, -3, -2, -1]
    x = np.arange(9.0).reshape(3, 3) + 0j
    assert np.array_equal(F.truncate_wrapped_to_centred(F.pad_centred_to_wrapped(x, [7, 8]), [3, 3]), x)
