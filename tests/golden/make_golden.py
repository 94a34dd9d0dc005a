"""Write reference bounds computed by the CPU oracle (only ``oracle/`` and the
seeded inputs of ``workloads/`` are used; nothing comes from the CUDA path).

The paper prints no bound for these synthetic microstructures; these values
are the oracle's FP64 Ga bounds (CG tolerance 1e-12, M = 2N - 1), stored so
the GPU tests need not rerun the slow oracle at moderate N.

    python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import coefficients as C  # noqa: E402
from oracle import galerkin as G  # noqa: E402

CASES = {
    "square_N15": lambda: W.centred_square(15),
    "disk_N81": lambda: W.centred_disk(81, fraction=0.3, value=100.0),
    "disk_N243": lambda: W.centred_disk(243, fraction=0.3, value=100.0),
    "disk_N729": lambda: W.centred_disk(729, fraction=0.3, value=100.0),
    "sphere_N33": lambda: W.centred_sphere(33, fraction=0.2, value=1000.0),
    "cube_N33": lambda: W.centred_cube(33, side=0.6, value=1000.0),
}


def main(names):
    out_dir = os.path.dirname(os.path.abspath(__file__))
    for name in names:
        m = CASES[name]()
        t0 = time.time()
        U, L, infos = G.bounds(C.material_from_dict(m), m["N"], tol=1e-12)
        rec = {"name": name, "microstructure": m, "tol": 1e-12, "M": [2 * n - 1 for n in m["N"]],
               "upper": U.tolist(), "lower": L.tolist(),
               "iters": {f"{k[0]}_{k[1]}": v["iters"] for k, v in infos.items()},
               "seconds": time.time() - t0,
               "source": "oracle/galerkin.py bounds() -- FP64 CPU oracle, not a paper value"}
        with open(os.path.join(out_dir, f"{name}.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(name, rec["seconds"], U.tolist(), L.tolist(), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["square_N15", "disk_N81", "disk_N243", "sphere_N33", "cube_N33"])
