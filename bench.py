"""Throughput of the Ga guaranteed-bounds hot path on GB300.

One step = one bound pair of the measured workload: rebuild the coefficient
tables a^, (1/a)^ on Z_{2N-1} and the double-grid values A_M, B_M from the
inclusion list, then d primal and d dual CG solves with FP64 residual
correction around FP32 inner iterations, the exact FP64 projection of every
minimiser and the FP64 Gram energies -> upper and lower d x d bounds.

Workload (default): d = 2, unit cell, one centred disk of volume fraction 0.3,
contrast 100 (inclusion 100, matrix 1), N = 2187 (double grid 4374 x 4374),
CG relative residual 1e-10; synthetic (seeded microstructure, nothing read).

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica on its own GPU (the solves shard by instance; no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "bound pairs/s & grid-pt·iter/s, mixed vs FP64 at 1e-8 rel err; p50/p99 latency"
UNIT = "bound pairs/s"
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA peak: 152 SMs x 4 FP64 flop/clk x 2.07 GHz (a plain FMA loop measured
# 1.20 TFLOP/s on this part)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=2187)
    ap.add_argument("--fp64-steps", type=int, default=1, help="steps of the plain FP64 path (comparison)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reduced-steps", type=int, default=1,
                    help="bound pairs timed with the reduced form of the operator (0 = skip)")
    ap.add_argument("--image-steps", type=int, default=1,
                    help="voxel-image bound pairs timed (0 = skip)")
    ap.add_argument("--image-N", type=int, default=99, help="order N of the voxel-image workload")
    ap.add_argument("--warm-steps", type=int, default=1,
                    help="run the coarse-to-fine start comparison (0 = skip)")
    ap.add_argument("--gani-steps", type=int, default=1,
                    help="GaNi a-posteriori bound pairs timed on the same workload (0 = skip)")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="instances of the batched workload (0 = skip)")
    ap.add_argument("--batch-sample", type=int, default=16,
                    help="randomly drawn instances on which the batched and the FP64 single-solve arms "
                         "are both timed")
    ap.add_argument("--d3-N", type=str, default="33,65,129",
                    help="orders of the d = 3 sphere / cube legs (comma list; empty = skip)")
    ap.add_argument("--d3-fp64-max-N", type=int, default=129,
                    help="largest d = 3 order also timed on the plain FP64 path")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="measured arrival window of the sustained served run (0 = skip the served leg)")
    ap.add_argument("--serve-warmup", type=float, default=2.0,
                    help="arrival window before the measured one (its requests are not counted)")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="sustained arrival rate as a fraction of the measured service capacity")
    ap.add_argument("--serve-probe", type=int, default=96,
                    help="requests of the closed-loop capacity probe (mixed; a quarter of it for FP64)")
    ap.add_argument("--serve-overload-rate", type=float, default=200.0,
                    help="arrival rate of the short overload run (0 = skip)")
    ap.add_argument("--serve-overload-seconds", type=float, default=2.0)
    ap.add_argument("--serve-overload-drain", type=float, default=10.0,
                    help="seconds after the overload run's last arrival before it stops waiting")
    ap.add_argument("--serve-drain", type=float, default=30.0,
                    help="seconds after the last arrival before a served run stops waiting")
    ap.add_argument("--serve-slots", type=int, default=64,
                    help="requests the server solves at once (more wait in its queue)")
    ap.add_argument("--serve-fp64-seconds", type=float, default=30.0,
                    help="measured arrival window of the plain FP64 served run (0 = skip)")
    ap.add_argument("--matvec-workload", choices=["disk", "sphere"], default="disk",
                    help="--matvec-only: the d = 2 disk (default) or the d = 3 sphere of volume fraction 0.2, "
                         "contrast 1000, at order --N")
    ap.add_argument("--matvec-only", choices=["f32", "f64"], default=None,
                    help="only apply the operator (warmup + steps times) at the workload size; "
                         "prints the mean time per application (used for ncu captures)")
    return ap.parse_args()


def workload(N):
    import workloads as W
    return W.centred_disk(N, fraction=0.3, value=100.0)


def workload_name(N):
    return f"d2 centred disk vf=0.3 contrast 100, N={N} (double grid {2 * N})"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import coefficients as C, galerkin as G
m = W.centred_disk({N}, fraction=0.3, value=100.0)
mat = C.material_from_dict(m)
t0 = time.perf_counter()
op = G.Operator(mat, m["N"], G.PRIMAL, M=[{M}, {M}])
t_setup = time.perf_counter() - t0
x = W.random_field(np.random.default_rng(1), 2, m["N"])
ts = []
for _ in range({reps}):
    t0 = time.perf_counter()
    op.apply(x)
    ts.append(time.perf_counter() - t0)
print(json.dumps(dict(setup_s=t_setup, matvec_s=ts)))
"""


def oracle_matvec_times(N, M, reps):
    """Run the oracle (single-threaded numpy) in a child process: set-up time
    and `reps` timed operator applications at the full workload size."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, N=N, M=M, reps=reps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# operator applications of one FP64 bound pair at the default workload:
# 2 primal + 2 dual CG solves (iterations measured on the FP64 GPU path, same
# algorithm and tolerance) plus one application per admissible field for the
# Gram energies.  Printed by the ours arm as "fp64.matvecs_per_pair".
FP64_MATVECS_PER_PAIR = {2187: 350}


def run_reference(args, world, rank):
    if rank != 0:
        return
    N = args.N
    M = 2 * N
    reps = max(1, args.steps)
    mv_pair = FP64_MATVECS_PER_PAIR.get(N)
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up state; warm-up steps are not timed
    res = oracle_matvec_times(N, M, reps)
    t = sum(res["matvec_s"]) / len(res["matvec_s"])
    mv = mv_pair if mv_pair else 4 * 100 + 4
    value = 1.0 / (t * mv)
    extrapolated = (f"extrapolated: {reps} oracle operator application(s) timed, x {mv} applications of one "
                    f"FP64 bound pair (the count the FP64 GPU path measures at this workload)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": reps, "warmup": args.warmup, "ms_per_step": 1e3 * t * mv, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(N), "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"{reps} oracle operator applications at N={N}, M={M} "
                                   f"(mean {t:.2f} s each), x {mv} applications per bound pair",
                         "extrapolation": extrapolated},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    t_bench0 = time.perf_counter()

    import paper_1412_2033_gb300 as g

    torch.cuda.set_device(local)
    g.load_library()
    m = workload(args.N)
    incs = m["inclusions"]

    ctx = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    for _ in range(args.warmup):
        ctx.set_coeffs(m["a0"], incs)
        ctx.bounds()

    # ---- timed region: K steps on resident buffers, CUDA events on the context's stream
    barrier(world)
    torch.cuda.synchronize()
    ctx.profile(True)
    lat = []
    U = L = infos = None
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.set_coeffs(m["a0"], incs)
            U, L, infos, st = ctx.bounds()
            e1.record(stream)
            lat.append((e0, e1))
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    elapsed = t_start.elapsed_time(t_end) / 1e3
    prof = ctx.profile_read()
    ctx.profile(False)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    elapsed_max = allmax(world, elapsed)
    pairs = args.steps * world
    value = pairs / elapsed_max

    iters32 = sum(i["matvecs_fp32"] for i in infos)
    iters64 = sum(i["matvecs_fp64"] for i in infos)
    grid_pts = float(np.prod(ctx.M))
    gpi = (iters32 + iters64 + 2 * m["d"]) * grid_pts * args.steps * world / elapsed_max

    # ---- roofline of the dominant kernel (from the live event timings above)
    hbm, peak_src = peaks()
    dom_name, dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    avg_s = dom["ms"] / dom["launches"] / 1e3
    f32 = dom_name.endswith("_f32")
    if f32 or dom["flops"] == 0:
        achieved = dom["bytes"] / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": peak_src}
    else:
        achieved = dom["flops"] / avg_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "derived FP64 FMA peak"}
    roof["kernel"] = dom_name
    roof["traffic"] = traffic_for(dom_name)
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "avg_us": round(1e3 * v["ms"] / v["launches"], 2),
                   "GBps": round(v["bytes"] / (v["ms"] / v["launches"] / 1e3) / 1e9, 1) if v["bytes"] else None,
                   "share": round(v["ms"] / sum(x["ms"] for x in prof.values()), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    launches = sum(v["launches"] for v in prof.values())

    # ---- plain FP64 path on the same workload (the comparison of the metric)
    fp64 = None
    if args.fp64_steps > 0:
        c64 = g.Context.from_microstructure(m, precision="fp64", tol=1e-10)
        c64.set_stream(stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fp64_steps):
            c64.set_coeffs(m["a0"], incs)
            U64, L64, inf64, _ = c64.bounds()
        torch.cuda.synchronize()
        t64 = (time.perf_counter() - t0) / args.fp64_steps
        mv64 = sum(i["matvecs_fp64"] for i in inf64) + 2 * m["d"]
        err_u = float(np.abs(U - U64).max() / np.abs(U64).max())
        err_l = float(np.abs(L - L64).max() / np.abs(L64).max())
        fp64 = {"bound_pairs_per_s": 1.0 / t64, "s_per_pair": t64, "matvecs_per_pair": mv64,
                "grid_pt_iter_per_s": grid_pts * mv64 / t64,
                "mixed_speedup": value / world / (1.0 / t64), "rel_err_upper": err_u, "rel_err_lower": err_l,
                "upper": U64.tolist(), "lower": L64.tolist()}
        c64.close()

    # ---- GaNi scheme on the same workload (a-posteriori guaranteed bounds, eq. GaNi_apost)
    gani = None
    if args.gani_steps > 0:
        cg = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
        cg.set_stream(stream)
        cg.bounds_gani()                      # builds the N-grid plans and samples
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.gani_steps):
            cg.set_coeffs(m["a0"], incs)
            GU, GL, GA, GB, ginf, _ = cg.bounds_gani()
        torch.cuda.synchronize()
        tg = (time.perf_counter() - t0) / args.gani_steps
        gani = {"bound_pairs_per_s": 1.0 / tg, "s_per_pair": tg,
                "cg_iterations_per_pair": sum(i["iters"] for i in ginf),
                "upper_apost": GU.tolist(), "lower_apost": GL.tolist(), "A_gani": GA.tolist(),
                "B_gani_inv": GB.tolist(),
                "ga_width": float(U[0][0] - L[0][0]), "gani_apost_width": float(GU[0][0] - GL[0][0]),
                "note": "mixed precision; Ga bounds lie inside the a-posteriori GaNi bounds"}
        cg.close()

    # ---- coarse-to-fine start (Section 7.4): the N/3 solution prolongated as the
    # initial guess of the fine primal solve, against the cold start
    warm = None
    if args.warm_steps > 0 and m["d"] == 2:
        Nc = args.N // 3 if (args.N // 3) % 2 == 1 else args.N // 3 + 1
        E = [1.0, 0.0]
        cfine = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
        ccoarse = g.Context.from_microstructure(dict(m, N=[Nc, Nc]), precision="mixed", tol=1e-10)
        for s_ in (cfine, ccoarse):
            s_.set_stream(stream)

        def warm_path():
            fc, icoarse, _, _ = ccoarse.solve_ex(E)
            ec = fc.clone()
            ec[0, (Nc - 1) // 2, 0] -= E[0]
            x0 = g.prolong(ec, [args.N, args.N])
            _, iwarm, ewarm, _ = cfine.solve_ex(E, x0=x0, energies=True)
            return icoarse, iwarm, ewarm

        # one untimed pass of both paths first (first launches of their kernels,
        # which the first process after a build loads from the library file)
        cfine.solve_ex(E, energies=True)
        warm_path()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, icold, ecold, _ = cfine.solve_ex(E, energies=True)
        torch.cuda.synchronize()
        t_cold = time.perf_counter() - t0
        t0 = time.perf_counter()
        icoarse, iwarm, ewarm = warm_path()
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t0
        warm = {"coarse_N": Nc, "cold": {"s": t_cold, "inner_iters": icold["iters"], "start_bound": ecold[0],
                                          "bound": icold["energy"]},
                "warm": {"s": t_warm, "coarse_inner_iters": icoarse["iters"], "inner_iters": iwarm["iters"],
                         "start_bound": ewarm[0], "bound": iwarm["energy"]},
                "note": "primal load e_1, mixed precision, relative residual 1e-10; start_bound = energy "
                        "of the initial field (Voigt for the cold start, the coarse bound for the warm one)"}
        cfine.close()
        ccoarse.close()

    # ---- reduced form of the operator (Algorithm 3) on the same workload
    reduced = None
    if args.reduced_steps > 0 and all(mm == 2 * nn for mm, nn in zip(ctx.M, m["N"])):
        cr = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
        cr.set_stream(stream)
        bytes_dg = cr.device_bytes()
        cr.set_form("reduced")
        cr.bounds()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.reduced_steps):
            cr.set_coeffs(m["a0"], incs)
            RU, RL, rinf, _ = cr.bounds()
        torch.cuda.synchronize()
        tr = (time.perf_counter() - t0) / args.reduced_steps
        reduced = {"bound_pairs_per_s": 1.0 / tr, "s_per_pair": tr,
                   "rel_diff_upper_vs_double_grid": float(np.abs(RU - U).max() / np.abs(U).max()),
                   "rel_diff_lower_vs_double_grid": float(np.abs(RL - L).max() / np.abs(L).max()),
                   "device_bytes_double_grid_only": bytes_dg, "device_bytes_with_reduced": cr.device_bytes(),
                   "note": "mixed precision; 2^d shifted N-size transforms per application (M = 2N)"}
        cr.close()

    # ---- grid-based composite: a 99^3 two-phase voxel image (Section 7.5 stand-in)
    image = None
    if args.image_steps > 0:
        import workloads as W
        img = W.voxel_foam(P=99)
        Ni = [args.image_N] * 3
        ci = g.Context.from_image(img, Ni, precision="mixed", tol=1e-10)
        ci.set_stream(stream)
        ci.bounds()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.image_steps):
            ci.set_image(img)
            IU, IL, iinf, _ = ci.bounds()
        torch.cuda.synchronize()
        ti = (time.perf_counter() - t0) / args.image_steps
        image = {"workload": f"seeded 99^3 two-phase voxel image (0.49 / 0.029, porosity "
                             f"{float((img < 0.1).mean()):.2f}), d = 3, N = {Ni}, M = {ci.M}",
                 "bound_pairs_per_s": 1.0 / ti, "s_per_pair": ti, "upper": IU.tolist(), "lower": IL.tolist(),
                 "cg_iterations_per_pair": sum(i["iters"] for i in iinf),
                 "note": "mixed precision; set-up (image DFTs, tables, double-grid values) inside each step"}
        ci.close()

    # ---- end to end through the public API: host inclusion list in, host bounds out
    e2e_ts = []
    phase_bytes = 64 * max(1, len(incs))
    out_bytes = 2 * m["d"] * m["d"] * 8
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
        c.bounds()
        c.close()
        e2e_ts.append(time.perf_counter() - t0)
    e2e_t = allmax(world, statistics.median(e2e_ts)) if e2e_ts else float("nan")

    d3 = run_d3(args, g, stream) if args.d3_N.strip() else None
    batched = run_batched(args, g) if args.batch_count > 0 else None
    served = run_served(args, g) if args.serve_seconds > 0 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            res = oracle_matvec_times(args.N, ctx.M[0], 1)
            t = res["matvec_s"][0]
            mvp = fp64["matvecs_per_pair"] if fp64 else 4 * 100 + 4
            cpu = {"value": 1.0 / (t * mvp), "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": f"1 oracle operator application at N={args.N}, M={ctx.M[0]} ({t:.1f} s, "
                             f"set-up {res['setup_s']:.1f} s) x {mvp} applications per FP64 bound pair "
                             f"(extrapolated from the one timed application)"}
        except Exception as ex:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {ex}"}

    if rank == 0:
        def r3(x):
            return None if x is None else float(f"{x:.3g}")

        # compact summary, printed last: a reader of the line's tail sees it
        summary = {"mixed": {"pairs_per_s": r3(value / world), "gpt_iter_per_s": r3(gpi / world)}}
        if fp64:
            summary["fp64"] = {"pairs_per_s": r3(fp64["bound_pairs_per_s"]),
                               "gpt_iter_per_s": r3(fp64["grid_pt_iter_per_s"])}
            summary["mixed_speedup"] = r3(fp64["mixed_speedup"])
            summary["rel_err_mixed_vs_fp64"] = r3(max(fp64["rel_err_upper"], fp64["rel_err_lower"]))
        if d3:
            summary["d3[mixed,fp64,speedup,rel_err]"] = {
                f'{c["shape"]}{c["N"]}': [r3(c.get(k)) for k in ("mixed_pairs_per_s", "fp64_pairs_per_s",
                                                                 "mixed_speedup", "rel_err_upper")]
                for c in d3["cases"]}
        if batched:
            summary["batched[pairs_s,x_fp64_single]"] = [r3(batched["bound_pairs_per_s"]),
                                                         r3(batched["sample"]["speedup_vs_fp64_single"])]
        if served:
            summary["served[rate,pairs_s,p50_ms,p99_ms]"] = {
                arm: [r3(served[arm]["rate_req_per_s"]), r3(served[arm]["bound_pairs_per_s"]),
                      r3(served[arm]["latency_ms"]["p50"]), r3(served[arm]["latency_ms"]["p99"])]
                for arm in ("mixed", "fp64", "overload") if arm in served}
        summary["roofline_frac"] = r3(roof["frac"])
        top = dict(list(kernels.items())[:8])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded microstructure; nothing read from disk)",
            "config": {"workload": workload_name(args.N), "N": [args.N, args.N], "M": ctx.M,
                       "precision": "mixed: FP32 inner CG, FP64 residual correction, FP64 projection and Gram",
                       "tol": 1e-10, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (per-step working set ~1.5 GB)"},
            "kernels_top": top,
            "bounds": {"upper": U.tolist(), "lower": L.tolist()},
            "grid_pt_iter_per_s": gpi,
            "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                            int(0.99 * len(lat_ms)))]},
            "fp64": fp64,
            "d3": d3,
            "batched": batched,
            "served": served,
            "gani": gani,
            "warm_start": warm,
            "reduced": reduced,
            "image": image,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": {"value": pairs / e2e_t / args.steps * args.steps if e2e_ts else None, "unit": UNIT,
                    "h2d_bytes_per_step": phase_bytes, "d2h_bytes_per_step": out_bytes,
                    "what": "ghb_create (device set-up from the host inclusion list) + ghb_bounds "
                            "(results to host) + ghb_destroy, host wall clock"},
            "cpu_baseline": cpu,
            "bench_wall_s": round(time.perf_counter() - t_bench0, 1),
            "roofline": roof,
            "summary": summary,
        }
        if line["e2e"]["value"] is not None:
            line["e2e"]["value"] = world / e2e_t
        print(json.dumps(line), flush=True)
    ctx.close()


def _auto_M(N):
    """The library's automatic double grid: the smallest M >= 2N - 1 whose
    prime factors are 2, 3 and 5."""
    M = 2 * N - 1
    while True:
        m = M
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            return M
        M += 1


def _grid_pt_iters(M, infos, d):
    """grid-pt.iter of one bound pair: |M| x operator applications (FP32 and
    FP64 iterations and corrections, plus one application per admissible field
    for the Gram energies)."""
    import numpy as np
    mv = sum(i["matvecs_fp32"] + i["matvecs_fp64"] for i in infos) + 2 * d
    return float(np.prod(M)) * mv


def run_batched(args, g):
    """The 512-instance workload: K ~ U{1..20} disks of radius U(0.03, 0.12),
    contrast log-uniform in [2, 1e4], N odd uniform in 31..255; all instances
    solved together by the batch engine (one launch per kernel and CG
    iteration over every active solve).  The batched and the plain FP64
    single-solve arms are also both timed on one randomly drawn sample of the
    same instances, and both report grid-pt.iter/s."""
    import numpy as np
    import torch

    import workloads as W
    inst = W.disk_batch(args.batch_count)

    def batched_run(items):
        b = g.Batch()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [b.submit(m) for m in items]
        b.run(iterations=8)
        t = time.perf_counter() - t0
        res = {r["id"]: r for r in b.results()}
        st = b.stats()
        b.close()
        return t, [res[i] for i in ids], st

    # the workload's transform lengths are tuned before the timed run, as a
    # server tunes its lengths once at start-up (untimed)
    for M in sorted({_auto_M(n) for m in inst for n in m["N"]}):
        g.tune_get(M)
    t, res, st = batched_run(inst)
    ok = sum(1 for r in res if r["status"] == 0)
    iters = [sum(i["iters"] for i in r["infos"]) for r in res]
    # the same randomly drawn sample through both arms
    rng = np.random.default_rng(20141206)
    pick = sorted(rng.choice(len(inst), size=min(args.batch_sample, len(inst)), replace=False).tolist())
    sample = [inst[k] for k in pick]
    tb, resb, _ = batched_run(sample)
    gpi_b = 0.0
    for m, r in zip(sample, resb):
        M = [_auto_M(n) for n in m["N"]]
        gpi_b += _grid_pt_iters(M, r["infos"], m["d"])
    errs = []
    t64 = 0.0
    gpi_64 = 0.0
    for m, r in zip(sample, resb):
        c = g.Context.from_microstructure(m, precision="fp64", tol=1e-10)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        U, L, inf64, _ = c.bounds()
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t1
        gpi_64 += _grid_pt_iters(c.M, inf64, m["d"])
        c.close()
        errs.append(max(float(np.abs(r["upper"] - U).max() / np.abs(U).max()),
                        float(np.abs(r["lower"] - L).max() / np.abs(L).max())))
    return {"workload": f"{len(inst)} seeded d2 disk instances, N odd 31..255, contrast 2..1e4",
            "bound_pairs_per_s": len(inst) / t, "seconds": t, "ok": ok,
            "cg_iterations_per_pair_mean": float(np.mean(iters)), "launches": st["launches"],
            "sample": {"instances": pick, "batched_pairs_per_s": len(sample) / tb,
                       "batched_grid_pt_iter_per_s": gpi_b / tb,
                       "fp64_single_solve_pairs_per_s": len(sample) / t64,
                       "fp64_single_solve_grid_pt_iter_per_s": gpi_64 / t64,
                       "speedup_vs_fp64_single": (len(sample) / tb) / (len(sample) / t64),
                       "max_rel_err_vs_fp64": max(errs) if errs else None,
                       "note": "both arms timed on the same seeded random sample of the 512 instances "
                               "(batched: submit to results; FP64: one context per instance, bounds only)"},
            "note": "the workload's transform lengths tuned before the timed run; the timed run is "
                    "submit of all 512 instances to their results"}


def _serve_stream(rate, seconds, seed):
    import workloads as W
    return W.request_stream(rate=rate, duration=seconds, seed=seed)


def _percentiles(lat):
    lat = sorted(lat)
    if not lat:
        return {"p50": None, "p99": None}
    return {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


def _serve_mixed(g, stream, slots, t_measure0, t_measure1, drain):
    """Feed (arrival, request) pairs into one batch as they arrive (continuous
    batching).  Returns latency stats of the requests that arrived inside
    [t_measure0, t_measure1) and the completion rate over the arrival window."""
    b = g.Batch(max_active=slots)
    t0 = time.perf_counter()
    arrivals, done = {}, {}
    i = 0
    deadline = (stream[-1][0] if stream else 0.0) + drain
    while (i < len(stream) or len(done) < i) and time.perf_counter() - t0 < deadline:
        now = time.perf_counter() - t0
        while i < len(stream) and stream[i][0] <= now:
            arrivals[b.submit(stream[i][1])] = stream[i][0]
            i += 1
        if len(done) < i:
            b.step(iterations=4)
            tnow = time.perf_counter() - t0
            for r in b.results():
                done[r["id"]] = (tnow, r["status"])
        else:
            time.sleep(0.0005)
    wall = time.perf_counter() - t0
    b.close()
    meas = [k for k, a in arrivals.items() if t_measure0 <= a < t_measure1]
    # requests still unfinished at the cutoff enter with their age at the cutoff
    lat = [(done[k][0] if k in done else wall) - arrivals[k] for k in meas]
    fin = [done[k][0] for k in meas if k in done]
    window = max(fin) - t_measure0 if fin else float("nan")
    return {"submitted": len(meas), "completed": len(fin), "unfinished_at_cutoff": len(meas) - len(fin),
            "latency_ms": _percentiles(lat), "mean_latency_ms": 1e3 * sum(lat) / len(lat) if lat else None,
            "bound_pairs_per_s": len(fin) / window if fin else 0.0, "wall_s": wall,
            "ok": sum(1 for k in meas if k in done and done[k][1] == 0)}


def _serve_fp64(g, stream, t_measure0, t_measure1, drain):
    """The plain FP64 single-solve server: requests in arrival order, one FP64
    context at a time (create, bounds, destroy)."""
    import torch
    t0 = time.perf_counter()
    lat, fin, n = [], [], 0
    deadline = (stream[-1][0] if stream else 0.0) + drain
    for a, m in stream:
        now = time.perf_counter() - t0
        if now > deadline:
            break
        if a > now:
            time.sleep(a - now)
        c = g.Context.from_microstructure(m, precision="fp64", tol=1e-10)
        c.bounds()
        c.close()
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        if t_measure0 <= a < t_measure1:
            n += 1
            lat.append(tf - a)
            fin.append(tf)
    wall = time.perf_counter() - t0
    meas = [a for a, _ in stream if t_measure0 <= a < t_measure1]
    # requests never started before the cutoff enter with their age at the cutoff
    lat += [wall - a for a in meas[n:]]
    window = max(fin) - t_measure0 if fin else float("nan")
    return {"submitted": len(meas), "completed": n, "unfinished_at_cutoff": len(meas) - n,
            "latency_ms": _percentiles(lat), "mean_latency_ms": 1e3 * sum(lat) / len(lat) if lat else None,
            "bound_pairs_per_s": n / window if fin else 0.0, "wall_s": wall}


def run_served(args, g):
    """Poisson arrivals of bound requests mixing d = 2 disk instances (N odd
    63..1023) and d = 3 sphere instances (N odd 15..129), 50/50.

    1. capacity: a closed-loop probe (all probe requests submitted at once)
       gives the service rate C of each arm;
    2. sustained: arrivals at load x C for a warm-up window plus the measured
       window; latency = arrival -> result (host clock) of the requests that
       arrived in the measured window, throughput = their completions / time;
    3. overload (mixed only): the 200 req/s stream for a short window, labelled
       as such -- one GPU does not sustain it, so its latencies are queueing.
    Mixed = the batch engine (continuous batching); FP64 = one plain FP64
    context per request, in arrival order."""
    import torch
    out = {"mix": "50% d2 disks N odd 63..1023 (contrast 2..1e4), 50% d3 spheres N odd 15..129 "
                  "(contrast 2..1e3)", "slots": args.serve_slots}
    # 1. capacity of the mixed arm (closed loop)
    probe = [m for _, m in _serve_stream(1e6, args.serve_probe / 1e6, 7)][: args.serve_probe]
    b = g.Batch(max_active=args.serve_slots)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in probe:
        b.submit(m)
    b.run(iterations=4)
    cap = len(probe) / (time.perf_counter() - t0)
    b.results()
    b.close()
    rate = args.serve_load * cap
    W0, W1 = args.serve_warmup, args.serve_warmup + args.serve_seconds
    st = _serve_stream(rate, W1, 11)
    out["mixed"] = {"capacity_pairs_per_s": cap, "probe_requests": len(probe), "rate_req_per_s": rate,
                    "measured_window_s": args.serve_seconds, "warmup_s": W0,
                    **_serve_mixed(g, st, args.serve_slots, W0, W1, args.serve_drain)}
    if args.serve_overload_rate > 0:
        so = _serve_stream(args.serve_overload_rate, args.serve_overload_seconds, 13)
        out["overload"] = {"rate_req_per_s": args.serve_overload_rate,
                           "window_s": args.serve_overload_seconds,
                           "note": "beyond one GPU's capacity: latencies are queueing times",
                           **_serve_mixed(g, so, args.serve_slots, 0.0, args.serve_overload_seconds,
                                          args.serve_overload_drain)}
    if args.serve_fp64_seconds > 0:
        probe64 = probe[: max(6, args.serve_probe // 8)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for m in probe64:
            c = g.Context.from_microstructure(m, precision="fp64", tol=1e-10)
            c.bounds()
            c.close()
        torch.cuda.synchronize()
        cap64 = len(probe64) / (time.perf_counter() - t0)
        rate64 = args.serve_load * cap64
        W1f = args.serve_warmup + args.serve_fp64_seconds
        s64 = _serve_stream(rate64, W1f, 17)
        out["fp64"] = {"capacity_pairs_per_s": cap64, "probe_requests": len(probe64), "rate_req_per_s": rate64,
                       "measured_window_s": args.serve_fp64_seconds, "warmup_s": W0,
                       **_serve_fp64(g, s64, W0, W1f, args.serve_drain)}
        out["mixed_vs_fp64_capacity"] = cap / cap64
    return out


def run_d3(args, g, stream):
    """d = 3 centred sphere (volume fraction 0.2) and centred cube (side 0.6),
    contrast 1000, at each order of --d3-N: bound pairs/s of the mixed path
    and of the plain FP64 path, their relative bound difference and
    grid-pt.iter/s; the axis-2 passes' roofline from the mixed run at the
    largest order."""
    import numpy as np
    import torch

    import workloads as W
    Ns = [int(x) for x in args.d3_N.split(",") if x.strip()]
    hbm, peak_src = peaks()
    out = {"workload": "d3 centred sphere vf 0.2 / centred cube side 0.6, contrast 1000, tol 1e-10",
           "cases": []}
    for shape in ("sphere", "cube"):
        for N in Ns:
            m = W.centred_sphere(N, fraction=0.2, value=1000.0) if shape == "sphere" else \
                W.centred_cube(N, side=0.6, value=1000.0)
            cm = g.Context.from_microstructure(m, precision="mixed", tol=1e-10)
            cm.set_stream(stream)
            cm.bounds()                            # first launches, plans
            prof = N == max(Ns) and shape == "sphere"
            torch.cuda.synchronize()
            if prof:
                cm.profile(True)
            t0 = time.perf_counter()
            U, L, inf, _ = cm.bounds()
            torch.cuda.synchronize()
            tm = time.perf_counter() - t0
            rec = {"shape": shape, "N": N, "M": cm.M, "mixed_pairs_per_s": 1.0 / tm,
                   "mixed_grid_pt_iter_per_s": _grid_pt_iters(cm.M, inf, 3) / tm,
                   "mixed_inner_iters": sum(i["iters"] for i in inf), "upper_00": U[0, 0], "lower_00": L[0, 0]}
            if prof:
                pr = cm.profile_read()
                cm.profile(False)
                roof = {}
                for k in ("col2_inv_f32", "col2_fwd_f32", "col1_inv_pupdate_f32", "row_matvec_f32", "col1_fwd_f32"):
                    v = pr.get(k)
                    if v and v["launches"]:
                        avg = v["ms"] / v["launches"] / 1e3
                        ach = v["bytes"] / avg / 1e9
                        roof[k] = {"avg_us": 1e6 * avg, "achieved_GBps": ach, "frac": ach / hbm}
                out["roofline_N%d" % N] = {"peak_GBps": hbm, "peak_source": peak_src, "kernels": roof}
            cm.close()
            if N <= args.d3_fp64_max_N:
                c64 = g.Context.from_microstructure(m, precision="fp64", tol=1e-10)
                c64.set_stream(stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                U64, L64, inf64, _ = c64.bounds()
                torch.cuda.synchronize()
                t64 = time.perf_counter() - t0
                c64.close()
                rec.update({"fp64_pairs_per_s": 1.0 / t64,
                            "fp64_grid_pt_iter_per_s": _grid_pt_iters(c64.M, inf64, 3) / t64,
                            "mixed_speedup": t64 / tm,
                            "rel_err_upper": float(np.abs(U - U64).max() / np.abs(U64).max()),
                            "rel_err_lower": float(np.abs(L - L64).max() / np.abs(L64).max())})
            out["cases"].append(rec)
    return out


def traffic_for(kernel_name):
    """DRAM bytes per launch of `kernel_name` from the committed ncu summary,
    or None when there is none or the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("sources_sha256") != sources_digest():
            return None
        return d.get("traffic_per_launch", {}).get(kernel_name)
    except Exception:  # noqa: BLE001
        return None


# the translation unit of the measured kernel (the FP32 last-axis pass at
# M = 4374) and every header it includes
TRAFFIC_SOURCES = ["paper_1412_2033_gb300/csrc/ct_4374.cu", "paper_1412_2033_gb300/csrc/passes_impl.cuh",
                   "paper_1412_2033_gb300/csrc/fft_ct.cuh", "paper_1412_2033_gb300/csrc/fft.cuh",
                   "paper_1412_2033_gb300/csrc/ghb_internal.cuh", "paper_1412_2033_gb300/csrc/reduce.cuh"]


def sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()


def run_matvec_only(args, local):
    import numpy as np
    import torch

    import paper_1412_2033_gb300 as g
    import workloads as W

    torch.cuda.set_device(local)
    m = workload(args.N) if args.matvec_workload == "disk" else W.centred_sphere(args.N, fraction=0.2, value=1000.0)
    ctx = g.Context.from_microstructure(m)
    dt = torch.complex64 if args.matvec_only == "f32" else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(g.half_from_full(
        W.random_field(np.random.default_rng(0), m["d"], m["N"])))).to(dt).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.matvec(x, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.matvec(x, out=y)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"matvec": args.matvec_only, "N": args.N, "M": ctx.M,
                      "ms_per_matvec": e0.elapsed_time(e1) / max(1, args.steps)}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.matvec_only:
        run_matvec_only(args, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
