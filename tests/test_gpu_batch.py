"""Batched and served solving (ghb_batch_*) on the GPU.

* every request's bounds equal the single-context mixed result and the FP64
  oracle (1e-8 relative, the mixed-path tolerance);
* a request gives the same bounds alone and inside a mix of other requests
  admitted at different times (continuous batching does not change a result);
* a request that cannot fit the device-memory budget is answered with
  GHB_ERR_OOM instead of blocking the queue.
"""
import numpy as np
import pytest

from conftest import one_sided_margins, one_sided_slack

import workloads as W
from oracle import coefficients as OC
from oracle import galerkin as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ghb():
    import paper_1412_2033_gb300 as g
    g.load_library()
    return g


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def requests():
    out = [W.random_disk_instance(W.BASE_SEED + i, N=n) for i, n in enumerate([15, 21, 33, 45, 31, 63])]
    out.append(W.random_sphere_instance(W.BASE_SEED + 50, N=9))
    out.append(W.random_sphere_instance(W.BASE_SEED + 51, N=11))
    out.append(W.centred_square(15))
    out.append(W.laminate(7, d=3, h=0.37, value=8.0, a0=1.5, center=0.11))
    return out


def test_batch_matches_single_and_oracle(ghb):
    reqs = requests()
    b = ghb.Batch()
    ids = [b.submit(m) for m in reqs]
    b.run(iterations=8)
    res = {r["id"]: r for r in b.results()}
    assert sorted(res) == sorted(ids)
    for rid, m in zip(ids, reqs):
        r = res[rid]
        assert r["status"] == 0, r
        ctx = ghb.Context.from_microstructure(m, precision="mixed")
        U, L, _, st = ctx.bounds()
        assert rel(r["upper"], U) < 1e-9 and rel(r["lower"], L) < 1e-9
        if m["d"] == 2 or m["N"][0] <= 9:
            Uo, Lo, _ = OG.bounds(OC.material_from_dict(m), m["N"], tol=1e-12)
            assert rel(r["upper"], Uo) < 1e-8 and rel(r["lower"], Lo) < 1e-8
            su, sl = one_sided_slack(m)
            mu, ml = one_sided_margins(r["upper"], r["lower"], Uo, Lo)
            assert mu >= -su and ml >= -sl, (mu, ml, su, sl)
    st = b.stats()
    assert st["active"] == 0 and st["pending"] == 0 and st["finished"] == len(reqs)
    b.close()


def test_alone_equals_in_mix(ghb):
    target = W.random_disk_instance(W.BASE_SEED + 99, N=41)
    alone = ghb.Batch()
    alone.submit(target)
    alone.run()
    ra = alone.results()[0]
    mix = ghb.Batch()
    others = [W.random_disk_instance(W.BASE_SEED + 200 + i, N=n) for i, n in enumerate([25, 61, 37, 17])]
    mix.submit(others[0])
    mix.submit(others[1])
    mix.step(iterations=4)                 # work in flight before the target arrives
    tid = mix.submit(target)
    mix.step(iterations=4)
    mix.submit(others[2])
    mix.submit(W.random_sphere_instance(W.BASE_SEED + 300, N=9))
    mix.run()
    rm = {r["id"]: r for r in mix.results()}[tid]
    assert rel(rm["upper"], ra["upper"]) < 1e-12 and rel(rm["lower"], ra["lower"]) < 1e-12


def test_request_larger_than_budget(ghb):
    b = ghb.Batch(budget_bytes=1 << 20)    # 1 MiB: no instance fits
    rid = b.submit(W.random_disk_instance(W.BASE_SEED + 7, N=63))
    b.run()
    r = b.results()[0]
    assert r["id"] == rid and r["status"] == 2          # GHB_ERR_OOM


def test_large_requests_beside_the_batch(ghb):
    """A request of at least 2^22 double-grid points (d = 3 at N = 81, M = 162)
    is solved by the large-request worker with a private context while the
    small ones run in the batched cycles: its bounds are those of a single
    context, the small ones' are unchanged, and the batch reports all of them."""
    big = W.random_sphere_instance(W.BASE_SEED + 61, N=81)
    small = [W.random_disk_instance(W.BASE_SEED + 62, N=45), W.random_sphere_instance(W.BASE_SEED + 63, N=11)]
    b = ghb.Batch()
    ids = [b.submit(small[0]), b.submit(big), b.submit(small[1])]
    st = b.stats()
    assert st["pending"] + st["active"] == 3
    b.run(iterations=8)
    res = {r["id"]: r for r in b.results()}
    assert sorted(res) == sorted(ids)
    assert b.stats()["finished"] == 3
    b.close()
    for rid, m in zip(ids, [small[0], big, small[1]]):
        r = res[rid]
        assert r["status"] == 0, r
        U, L, _, _ = ghb.Context.from_microstructure(m, precision="mixed").bounds()
        tol = 1e-13 if m is big else 1e-9
        assert rel(r["upper"], U) < tol and rel(r["lower"], L) < tol
