"""Pins of the grid-based composites (Lemma grid_compos, Remark eval_with_FFT).

* a block of pixels is a box: the image table equals the inclusion-matrix
  table of the same box (Remark anal_Fourier), centred or shifted, for images
  coarser and finer than Z_{2N-1};
* a constant image has the table a0 delta;
* a pixel laminate: the Ga bounds bracket its homogenised matrix (arithmetic
  mean of the pixel values along the layers, harmonic across) and tighten as
  N grows."""
import numpy as np
import pytest

from oracle import coefficients as C
from oracle import galerkin as G
from oracle import image as I


@pytest.mark.parametrize("P,N,shift", [([15, 9], [7, 7], (0, 0)), ([15, 9], [7, 7], (2, -3)),
                                       ([5, 7], [9, 11], (1, 2)), ([6, 8, 5], [5, 3, 5], (1, 0, 2))])
def test_pixel_block_is_a_box(P, N, shift):
    d = len(P)
    img = np.full(P, 2.0)
    block = np.ix_(*[np.mod(np.arange(-1, 2) + shift[a], P[a]) for a in range(d)])
    img[block] = 7.0
    box = C.Material(d, 2.0, [C.Inclusion(C.BOX, tuple(shift[a] / P[a] for a in range(d)),
                                          tuple(3.0 / P[a] for a in range(d)), 7.0)])
    ref = C.coeff_table(box, N)
    got = I.image_table(img, N)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_constant_image():
    t = I.image_table(np.full((4, 6), 3.5), [5, 5])
    z = np.zeros_like(t)
    z[4, 4] = 3.5
    assert np.abs(t - z).max() < 1e-14


def test_pixel_laminate_bounds():
    vals = np.array([1.0, 4.0, 9.0, 2.0, 30.0])
    img = np.repeat(vals[:, None], 4, axis=1)           # P = (5, 4), layers normal to e_1
    harm, arith = 1.0 / np.mean(1.0 / vals), np.mean(vals)
    prev = None
    for N in (5, 9, 15):
        up, lo = I.image_bounds(img, [N, N], tol=1e-12)
        assert lo[0, 0] <= harm * (1 + 1e-12) <= up[0, 0] * (1 + 2e-12)
        assert abs(up[1, 1] - arith) < 1e-10 * arith and lo[1, 1] <= arith * (1 + 1e-12)
        if prev is not None:
            assert up[0, 0] <= prev[0][0, 0] * (1 + 1e-12) and lo[0, 0] >= prev[1][0, 0] * (1 - 1e-12)
        prev = (up, lo)
