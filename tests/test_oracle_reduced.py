"""Pin of the reduced Ga operator (Lemma reduce_grid, Algorithm 3): with the
double grid M = 2N it equals the double-grid operator (Algorithm 2, itself
pinned against the dense Galerkin matrix), projected or not, primal or dual,
2-D and 3-D, square and ragged N; a wrong phase sign or a wrong sub-grid
offset breaks the equality."""
import numpy as np
import pytest

from oracle import coefficients as C
from oracle import galerkin as G


@pytest.mark.parametrize("N", [[5, 5], [7, 3], [3, 5, 3]])
@pytest.mark.parametrize("kind", [G.PRIMAL, G.DUAL, None])
def test_reduced_equals_double_grid(N, kind):
    rng = np.random.default_rng(sum(N) + (0 if kind is None else len(kind)))
    d = len(N)
    incs = [C.Inclusion(C.BOX, tuple(rng.uniform(-0.5, 0.5, 3)), tuple(rng.uniform(0.2, 0.6, 3)), 6.0)]
    if d == 2:
        incs.append(C.Inclusion(C.DISK, (0.3, -0.3, 0), (0.12,), 0.3))
    mat = C.Material(d, 1.7, incs)
    M = [2 * n for n in N]
    table = C.coeff_table(mat, N)
    aM = G.double_grid_values(table, M)
    x = rng.standard_normal((d,) + tuple(N)) + 1j * rng.standard_normal((d,) + tuple(N))
    ref = G.matvec_double_grid(x, aM, kind)
    got = G.reduced_matvec(x, aM, kind)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_wrong_shift_sign_is_caught():
    """Flipping the phase sign breaks the identity (the check has teeth)."""
    N = [5, 5]
    mat = C.Material(2, 1.0, [C.Inclusion(C.DISK, (0.1, 0.0, 0), (0.3,), 9.0)])
    aM = G.double_grid_values(C.coeff_table(mat, N), [10, 10])
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 5)) + 1j * rng.standard_normal((2, 5, 5))
    ref = G.matvec_double_grid(x, aM, None)
    flipped = G.reduced_matvec(x, aM[::-1, ::-1].copy(), None)     # values at -x instead of x
    assert np.abs(flipped - ref).max() > 1e-3 * np.abs(ref).max()
