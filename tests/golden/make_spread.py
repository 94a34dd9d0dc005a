"""Measure the CPU oracle's own spread between admissible double grids at the
largest contrasts of the batched workload (about 1e4), and write it to
tests/golden/oracle_spread.json (only ``oracle/`` and ``workloads/`` are used).

Any M >= 2N - 1 gives the same bilinear form (Lemma integ_eval_VM), so the
bounds the oracle computes at different M differ only by FP64 rounding; that
difference is the resolution of the oracle as a reference.  For each of the
eight largest-contrast instances of the 512-instance batch (at N = 31..45) the
bounds are computed at M = 2N - 1, at the smallest 5-smooth M >= 2N - 1 and at
M = 2N, and the largest relative difference of the diagonal entries is kept.
The one-sided checks of the GPU tests on instances of that contrast derive
their slack from the largest spread measured here.

    python tests/golden/make_spread.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import coefficients as C  # noqa: E402
from oracle import galerkin as G  # noqa: E402


def smooth(n):
    m = n
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def main():
    order = sorted(range(512), key=lambda i: -W.random_disk_instance(W.BASE_SEED + i)["inclusions"][0][3])[:8]
    recs = []
    for k, i in enumerate(order):
        m = W.random_disk_instance(W.BASE_SEED + i, N=31 + 2 * k)
        mat = C.material_from_dict(m)
        N = m["N"]
        Ms = sorted({2 * N[0] - 1, smooth(2 * N[0] - 1), 2 * N[0]})
        U, L = {}, {}
        for M in Ms:
            u, l, _ = G.bounds(mat, N, M=[M, M], tol=1e-12)
            U[M], L[M] = np.diag(u), np.diag(l)
        su = max(float(np.max(np.abs(U[a] - U[b]) / np.abs(U[b]))) for a in Ms for b in Ms)
        sl = max(float(np.max(np.abs(L[a] - L[b]) / np.abs(L[b]))) for a in Ms for b in Ms)
        recs.append({"batch_index": i, "N": N[0], "M": Ms, "contrast": m["inclusions"][0][3],
                     "spread_upper": su, "spread_lower": sl})
        print(recs[-1], flush=True)
    out = {"what": "largest relative difference of the oracle's diagonal bounds between admissible M",
           "instances": recs,
           "max_spread": max(max(r["spread_upper"], r["spread_lower"]) for r in recs),
           "source": "tests/golden/make_spread.py -- FP64 CPU oracle only"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_spread.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("max spread", out["max_spread"])


if __name__ == "__main__":
    main()
