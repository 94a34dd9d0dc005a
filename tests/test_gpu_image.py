"""GPU parity of grid-based (pixel image) composites (Lemma grid_compos,
Remark eval_with_FFT) against the oracle (oracle/image.py).

Tolerances: tables 1e-13 of the largest entry (FP64 DFTs of the image and
sinc factors); FP64 bounds 1e-12 relative; mixed bounds 1e-8 relative with
the one-sided checks of the inclusion path."""
import numpy as np
import pytest

import workloads as W
from oracle import image as OI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def image(P, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(0.0, np.log(100.0), P))    # contrast up to 100


CASES = [((20, 15), [9, 11]), ((7, 30), [15, 5]), ((6, 8, 5), [5, 3, 5]), ((12, 10, 9), [7, 7, 5])]


@pytest.mark.parametrize("P,N", CASES)
def test_image_tables(ghb, P, N):
    img = image(P, sum(P))
    ctx = ghb.Context.from_image(img, N)
    for kind, src in [(ghb.GHB_PRIMAL, img), (ghb.GHB_DUAL, 1.0 / img)]:
        ref = OI.image_table(src, N)[..., N[-1] - 1:]
        got = ctx.table(kind).cpu().numpy()
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("P,N", CASES[:3])
def test_image_bounds_fp64_and_mixed(ghb, P, N):
    img = image(P, 3 + sum(N))
    up, lo = OI.image_bounds(img, N, tol=1e-12)
    U, L, _, st = ghb.Context.from_image(img, N, tol=1e-12).bounds()
    assert st == 0 and rel(U, up) < 1e-12 and rel(L, lo) < 1e-12
    Um, Lm, _, st = ghb.Context.from_image(img, N, precision="mixed").bounds()
    assert st == 0 and rel(Um, up) < 1e-8 and rel(Lm, lo) < 1e-8
    s = 1e-13 * 100
    assert np.all(np.diag(Um) >= np.diag(up) * (1 - s)) and np.all(np.diag(Lm) <= np.diag(lo) * (1 + s))


def test_pixel_block_equals_box_on_gpu(ghb):
    P, N = (15, 9), [21, 17]
    img = np.full(P, 2.0)
    img[np.ix_([14, 0, 1], [8, 0, 1])] = 7.0
    m = dict(d=2, N=N, a0=2.0, inclusions=[(0, (0.0, 0.0, 0.0), (3 / 15, 3 / 9, 1.0), 7.0)])
    Ui, Li, _, _ = ghb.Context.from_image(img, N).bounds()
    Ub, Lb, _, _ = ghb.Context.from_microstructure(m).bounds()
    assert rel(Ui, Ub) < 1e-12 and rel(Li, Lb) < 1e-12


def test_image_context_switches(ghb):
    m = W.random_disk_instance(6, N=15)
    ctx = ghb.Context.from_image(image((10, 10), 1), [15, 15])
    with pytest.raises(ghb.GhbError):
        ctx.bounds_gani()                            # GaNi samples need inclusions
    ctx.set_coeffs(m["a0"], m["inclusions"])
    U, L, _, _ = ctx.bounds()
    U2, L2, _, _ = ghb.Context.from_microstructure(m).bounds()
    assert rel(U, U2) < 1e-13 and rel(L, L2) < 1e-13
    ctx.bounds_gani()                                # available again
