"""Write reference bounds computed by the CPU oracle (only ``oracle/`` and the
seeded inputs of ``workloads/`` are used; nothing comes from the CUDA path).

The paper prints no bound for these synthetic microstructures; these values
are the oracle's FP64 Ga bounds, stored so the GPU tests need not rerun the
slow oracle.  Each case fixes its double grid M (any M >= 2N - 1 gives the same
bilinear form, Lemma integ_eval_VM), its CG tolerance and, for the cases named
``*_k<K>``, a fixed number K of CG iterations: those store the bounds of the
K-th CG iterate (still guaranteed bounds, Def. Ga: any admissible field gives
one) at sizes where a converged oracle solve takes hours.

    python tests/golden/make_golden.py [--workers W] [name ...]

The 2d solves of a case (and the cases themselves) run in parallel in a
process pool of W workers (started with ``spawn``).
"""
import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import coefficients as C  # noqa: E402
from oracle import galerkin as G  # noqa: E402


def _high_contrast_batch_instance(N):
    """The instance of the 512-instance disk batch with the largest contrast,
    at order N (the batch's largest)."""
    best = max(range(512), key=lambda i: W.random_disk_instance(W.BASE_SEED + i)["inclusions"][0][3])
    return W.random_disk_instance(W.BASE_SEED + best, N=N)


def _m2(N):
    return [2 * n - 1 for n in N]


# name -> (microstructure, M or None for 2N - 1, tol, maxiter)
CASES = {
    "square_N15": lambda: (W.centred_square(15), None, 1e-12, 10000),
    "disk_N81": lambda: (W.centred_disk(81, fraction=0.3, value=100.0), None, 1e-12, 10000),
    "disk_N243": lambda: (W.centred_disk(243, fraction=0.3, value=100.0), None, 1e-12, 10000),
    "disk_N729": lambda: (W.centred_disk(729, fraction=0.3, value=100.0), None, 1e-12, 10000),
    "disk_N2187": lambda: (W.centred_disk(2187, fraction=0.3, value=100.0), [4374, 4374], 1e-12, 10000),
    "sphere_N33": lambda: (W.centred_sphere(33, fraction=0.2, value=1000.0), None, 1e-12, 10000),
    "cube_N33": lambda: (W.centred_cube(33, side=0.6, value=1000.0), None, 1e-12, 10000),
    "sphere_N65": lambda: (W.centred_sphere(65, fraction=0.2, value=1000.0), [135] * 3, 1e-12, 10000),
    "cube_N65": lambda: (W.centred_cube(65, side=0.6, value=1000.0), [135] * 3, 1e-12, 10000),
    "sphere_N129_k24": lambda: (W.centred_sphere(129, fraction=0.2, value=1000.0), [270] * 3, 1e-30, 24),
    "cube_N129_k24": lambda: (W.centred_cube(129, side=0.6, value=1000.0), [270] * 3, 1e-30, 24),
    "batch_maxcontrast_N255": lambda: (_high_contrast_batch_instance(255), None, 1e-12, 10000),
}
DEFAULT = list(CASES)


def run_case(name, pool, out_dir):
    m, M, tol, maxiter = CASES[name]()
    t0 = time.time()
    U, L, infos = G.bounds(C.material_from_dict(m), m["N"], M=M, tol=tol, maxiter=maxiter, pool=pool)
    rec = {"name": name, "microstructure": m, "tol": tol, "maxiter": maxiter,
           "M": M if M is not None else _m2(m["N"]),
           "upper": U.tolist(), "lower": L.tolist(),
           "iters": {f"{k[0]}_{k[1]}": v["iters"] for k, v in infos.items()},
           "relres": {f"{k[0]}_{k[1]}": v["relres"] for k, v in infos.items()},
           "seconds": time.time() - t0,
           "source": "oracle/galerkin.py bounds() -- FP64 CPU oracle, not a paper value"}
    with open(os.path.join(out_dir, f"{name}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(name, round(rec["seconds"], 1), U.tolist(), L.tolist(), flush=True)


def main(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=1)
    ap.add_argument("names", nargs="*")
    args = ap.parse_args(argv)
    names = args.names or DEFAULT
    out_dir = os.path.dirname(os.path.abspath(__file__))
    if args.workers <= 1:
        for n in names:
            run_case(n, None, out_dir)
        return
    with cf.ProcessPoolExecutor(max_workers=args.workers, mp_context=mp.get_context("spawn")) as pool:
        with cf.ThreadPoolExecutor(max_workers=len(names)) as cases:
            for fut in [cases.submit(run_case, n, pool, out_dir) for n in names]:
                fut.result()


if __name__ == "__main__":
    main(sys.argv[1:])
