#!/usr/bin/env python3
"""Benchmark of the AMG-preconditioned CG solve on one GB300.

Headline workload (the largest single-GPU configuration): 3D cell-centred
finite volumes, 512^3 cells (134,217,728 unknowns), diagonal anisotropic
coefficient K = exp(Z) diag(1, 1, 1e-3) with Z a Gaussian field (variance 6,
correlation length 0.02, 1000 cosine modes, seed 0), u = 1 at x = 0, u = 0 at
x = 1, no flux elsewhere.  A step is one complete solve to a 1e-8 relative
residual (every V-cycle and CG operation) with the hierarchy resident in HBM.

Metric: time to a 1e-8 relative residual (ms, lower is better) of FP64
AMG-PCG; the FP32-in-FP64 solve of the same system (time, iterations, distance
to the FP64 solution) and the V-cycle HBM bandwidth of both precisions are
reported beside it.  The same block is measured on the 256^3 layered workload
(log-normal K, variance 4, with 8 slabs of contrast 1e6) and on the 128^3
log-normal workload (variance 4, correlation length 0.05) under
"other_workloads".  Per-kernel records go to a file (--kernels-out), not to
the JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank solves its own replica on its own GPU with no
communication on the data path; timing is the maximum over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("time to 1e-8 relative residual, FP64 AMG-PCG (FP32-in-FP64 and V-cycle HBM GB/s "
          "beside it)")
UNIT = "ms"

# The configurations of the benchmark: name -> (description, default grid, maker)
WORKLOADS = {
    "anisotropic512": ("3D FV 7-point {g}^3 anisotropic K = exp(Z) diag(1,1,1e-3), Z variance 6, "
                       "correlation length 0.02; AMG-PCG to 1e-8, FP64 and FP32-in-FP64", 512),
    "layered256": ("3D FV 7-point {g}^3 log-normal K (variance 4, correlation length 0.05) with 8 "
                   "horizontal layers of contrast 1e6; AMG-PCG to 1e-8, FP64 and FP32-in-FP64", 256),
    "lognormal128": ("3D FV 7-point {g}^3 log-normal K (variance 4, correlation length 0.05); "
                     "AMG-PCG to 1e-8, FP64 and FP32-in-FP64", 128),
}


def make_problem(workload: str, grid: int):
    from paper_1209_0960_gb300 import problems
    g = (grid, grid, grid)
    if workload == "anisotropic512":
        return problems.anisotropic3d(g, variance=6.0, corr_len=0.02, zfac=1e-3, seed=0)
    if workload == "layered256":
        return problems.layered3d(g, seed=0)
    if workload == "lognormal128":
        return problems.lognormal3d(g, variance=4.0, corr_len=0.05, seed=0)
    raise KeyError(workload)


def fv7_nnz(grid: int) -> int:
    """Stored entries of the 7-point matrix on a grid^3 box: 7 per cell minus
    the two missing couplings of every boundary face pair."""
    return 7 * grid ** 3 - 6 * grid ** 2


def workload_config(args, workload: str, grid: int, world: int) -> dict:
    n = grid ** 3
    nnz = fv7_nnz(grid)
    return {"workload": WORKLOADS[workload][0].format(g=grid), "grid": grid, "unknowns": n,
            "nnz": nnz, "tol": args.tol,
            "l2": "inputs larger than L2 (level-0 matrix %.0f MB > 129 MB)" % ((nnz * 12 + 4 * n) / 1e6),
            "parallelism": f"replicas x{world}"}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="anisotropic512",
                    help="headline workload")
    ap.add_argument("--grid", type=int, default=0,
                    help="cells per axis of the headline workload (0: the workload's own)")
    ap.add_argument("--others", type=str, default="layered256,lognormal128",
                    help="comma-separated secondary workloads measured after the headline "
                         "('' for none)")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--cpu-grid", type=int, default=64,
                    help="cells per axis of the oracle's sample of the headline workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="timed steps of the end-to-end leg (at most --steps)")
    ap.add_argument("--kernels-out", type=str, default=os.path.join("gpurun_out", "bench_kernels.json"),
                    help="file for the per-kernel records of the profiled solves")
    ap.add_argument("--launch-overlap", type=int, choices=[0, 1], default=1,
                    help="programmatic dependent launch between solve kernels")
    ap.add_argument("--profile-run", type=int, default=0, metavar="MAXIT",
                    help="for profilers: set up the workload, run one solve capped at "
                         "MAXIT iterations, print nothing else and exit")
    ap.add_argument("--profile-fp32", action="store_true",
                    help="with --profile-run: the FP32-in-FP64 solve instead of FP64")
    ap.add_argument("--serving", type=int, default=0, metavar="N",
                    help="serving workload instead: N independent requests (box sides "
                         "U{16..96}, variance U[1,6]) with Poisson arrivals at --load times the "
                         "measured saturated rate; prints its own JSON line")
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--rate", type=float, default=0.0,
                    help="offered requests/s of the Poisson phase (0: --load times the saturated rate)")
    ap.add_argument("--host-threads", type=int, default=0,
                    help="host threads per setup for tiled aggregation (0: all host cores)")
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--batch-vcycles", type=int, choices=[0, 1], default=0,
                    help="serving: 1 runs the V-cycles of the requests that need one in a "
                         "scheduler tick as shared launches, level by level; 0: each request "
                         "launches its own")
    ap.add_argument("--serving-requests", type=int, default=200, metavar="N",
                    help="the bounded serving leg of the main line (0: none)")
    ap.add_argument("--setup-threads", type=int, default=0,
                    help="server setup threads (0: host cores - 3)")
    ap.add_argument("--aggregation-tile", type=int, default=-1, metavar="T",
                    help="decoupled aggregation (Alg. 4) in tiles of T consecutive rows "
                         "(0: Algorithm 1 over whole levels; default 0, and 4096 with --serving)")
    ap.add_argument("--device-loop", type=int, choices=[0, 1], default=None,
                    help="1: run the PCG iteration loop as one graph with a device-side WHILE node "
                         "(the solve default); 0: the host launches each iteration (same kernels, "
                         "same order; the serving default)")
    ap.add_argument("--coarsest-fp32", type=int, choices=[0, 1], default=0,
                    help="float32 V-cycle: apply the coarsest inverse as a float32 matrix "
                         "(default 0: float64 matrix)")
    ap.add_argument("--autotune", type=int, choices=[0, 1], default=1,
                    help="time the launch shapes of every level at setup and keep the fastest "
                         "(0: the fixed rules)")
    ap.add_argument("--coarsen-target", type=int, default=0, metavar="N",
                    help="stop coarsening at N rows (0: the library default)")
    ap.add_argument("--lanes-per-row", type=str, default="", metavar="L0,L1,...",
                    help="fixed launch shapes per level instead of tuning (0 = staged "
                         "kernels, else 1/2/4/8 lanes per row, with a suffix h for blocks of "
                         "128 threads and s for one dependency-driven kernel per smoothing "
                         "sweep; staged levels may add cP for a shared-memory carveout of P "
                         "percent, e.g. 0,0c58,2h,4hs), for reproducible profiles")
    ap.add_argument("--aggregation-device", type=int, choices=[0, 1], default=0,
                    help="with --aggregation-tile: run the tiles on the GPU (1) or on host threads")
    args = ap.parse_args()
    try:
        args.lanes = parse_lanes(args.lanes_per_row)
    except ValueError as e:
        ap.error(str(e))
    if args.lanes:
        args.autotune = 0
    if args.aggregation_tile < 0:
        args.aggregation_tile = 4096 if args.serving > 0 else 0
    if args.grid <= 0:
        args.grid = WORKLOADS[args.workload][1]
    args.others = [w.strip() for w in args.others.split(",") if w.strip()]
    for w in args.others:
        if w not in WORKLOADS:
            ap.error(f"unknown workload {w}")
    return args


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            import torch
            from datetime import timedelta
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            # a rank that dies makes the others' next collective fail within
            # this time instead of waiting forever
            timeout = float(os.environ.get("BENCH_PG_TIMEOUT_S", "900"))
            dist.init_process_group(backend, timeout=timedelta(seconds=timeout))
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if self.pg is None:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            sel = str(device_index)
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", sel, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
            os.unlink(self.path)
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        loaded = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_traffic(name: str, workload: str):
    """DRAM bytes per launch of kernel class `name` on `workload` from the
    committed ncu summary, if the kernel source has not changed since it was
    captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        rec = d[workload][name]
        src = open(os.path.join(ROOT, "paper_1209_0960_gb300", "csrc", rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec["sha256_16"]:
            return None
        return float(rec["bytes_per_launch"])
    except Exception:
        return None


def r4(v):
    """Round floats to 4 significant digits, recursively (keeps the line short)."""
    if isinstance(v, float):
        return float(f"{v:.4g}")
    if isinstance(v, dict):
        return {k: r4(x) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [r4(x) for x in v]
    return v


def oracle_sample(workload: str, grid: int, tol: float, steps: int, warmup: int,
                  min_seconds: float = 0.0, openmp: bool = False):
    """Time the oracle's PCG solve on the grid^3 instance of the workload (the
    serial build, or the OpenMP build of the same source on all host cores),
    hierarchy built once.  Returns a dict of seconds, iterations and sizes."""
    from oracle import oracle as O
    p = make_problem(workload, grid)
    t0 = time.perf_counter()
    H = O.Hierarchy(p.row_ptr, p.col, p.val, O.default_params(3), openmp=openmp)
    setup_s = time.perf_counter() - t0
    for _ in range(warmup):
        H.pcg(p.b, tol=tol, maxit=1000)
    times, it = [], 0
    t_all = time.perf_counter()
    while len(times) < steps or (time.perf_counter() - t_all) < min_seconds:
        t0 = time.perf_counter()
        _, it, _, _ = H.pcg(p.b, tol=tol, maxit=1000)
        times.append(time.perf_counter() - t0)
    return {"solve_s": statistics.mean(times), "iterations": it, "n": p.n, "solves": len(times),
            "setup_s": setup_s, "levels": H.num_levels, "problem": p}


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, dist: Dist):
    if dist.rank != 0:
        return
    smp = oracle_sample(args.workload, args.cpu_grid, args.tol, max(1, args.steps), args.warmup)
    value = smp["solve_s"] * 1e3
    sample = (f"oracle PCG solve (single thread) on the {args.cpu_grid}^3 instance of the workload "
              f"({smp['n']} unknowns, {smp['levels']} levels, {smp['iterations']} iterations), "
              f"hierarchy built once ({smp['setup_s']:.1f} s, not timed); unscaled: at "
              f"{smp['setup_s'] / smp['n'] * 1e6:.0f} us of setup a row, the oracle's setup of the "
              f"{args.grid}^3 system alone would take about "
              f"{smp['setup_s'] / smp['n'] * args.grid ** 3 / 60:.0f} min")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": smp["solves"], "warmup": args.warmup, "ms_per_step": value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, args.workload, args.grid, dist.world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "setup_s": smp["setup_s"], "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(r4(line)), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

VCYCLE_KINDS = {"gs_level0", "first_level0", "gs_coarse", "residual_level0",
                "residual_coarse", "restrict", "prolong", "coarse_solve", "zero", "convert"}


def timed_solves(solver, b, x, steps, tol, stream, dist, maxit):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    infos = []
    for _ in range(steps):
        x.zero_()
        _, rc, info = solver.solve(b, x, tol=tol, maxit=maxit)
        infos.append((rc, info))
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    return ev0.elapsed_time(ev1) / steps, infos


def parse_lanes(text: str) -> list:
    """--lanes-per-row text -> [(lanes_per_row, threads_per_block, carveout or None)]."""
    out = []
    for v in (v.strip() for v in text.split(",")):
        if v:
            m = re.fullmatch(r"(\d+)(h?)(s?)(?:c(\d+))?", v)
            if not m:
                raise ValueError(f"--lanes-per-row: cannot read {v!r}")
            lanes = int(m.group(1))
            if m.group(3):
                lanes |= 0x100   # AMG_SHAPE_SWEEP: one dependency-driven kernel per sweep
            carve = int(m.group(4)) if m.group(4) else None
            out.append((lanes, 128 if m.group(2) else 0, carve))
    return out


def apply_lanes(solver, args):
    for l, (lanes, threads, carve) in enumerate(args.lanes):
        solver.set_level_shape(l, lanes, threads)
        if carve is not None:
            solver.set_level_carveout(l, carve)


def shape_string(levels):
    """The levels' launch shapes in --lanes-per-row syntax."""
    out = []
    for lv in levels[:-1]:
        v = str(lv["lanes_per_row"]) + ("h" if lv["threads_per_block"] == 128 else "")
        v += "s" if lv["sweep"] else ""
        v += f"c{lv['carveout']}" if lv["carveout"] >= 0 else ""
        out.append(v)
    return ",".join(out)


def new_solver(args, p, stream):
    from paper_1209_0960_gb300 import amg
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, stream=stream,
                     launch_overlap=args.launch_overlap, aggregation_tile=args.aggregation_tile,
                     aggregation_device=args.aggregation_device, autotune=args.autotune,
                     coarsest_fp32=args.coarsest_fp32,
                     device_loop=1 if args.device_loop is None else args.device_loop,
                     **({"coarsen_target": args.coarsen_target} if args.coarsen_target else {}))
    apply_lanes(solver, args)
    return solver


def prof_iters(prof):
    return max([d["launches"] for d in prof if d["name"] == "coarse_solve"] or [1])


def measure_workload(args, dist, workload, grid, steps, warmup, headline, kernels_out):
    """Set up one workload and time K FP64 and K FP32-in-FP64 solves; with
    `headline` also the end-to-end leg, clocks and the roofline.  Returns the
    compact record and the per-kernel records."""
    import numpy as np
    import torch
    from paper_1209_0960_gb300 import amg

    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    p = make_problem(workload, grid)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    solver = new_solver(args, p, stream)
    setup_wall = time.perf_counter() - t0
    summary, levels = solver.info()
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    maxit = 1000
    peak, peak_src = measured_peaks()
    out = {}
    kern = {}

    def vcycle_gbs(graph_ms, model_bytes, cg_extra_bytes):
        gms = graph_ms.get("graph_vcycle_part")
        if not gms:
            return None
        wall = (model_bytes + cg_extra_bytes) / (gms * 1e-3) / 1e9
        return {"ms": gms, "gbs": wall, "frac_measured": wall / peak, "frac_nominal_7900": wall / 7900.0}

    res = {}
    clk = None
    for prec, tag in ((amg.AMG_FP64, "fp64"), (amg.AMG_FP32_IN_FP64, "fp32")):
        solver.set_precision(prec)
        for _ in range(warmup):
            x.zero_()
            solver.solve(b, x, tol=args.tol, maxit=maxit)
        clocks = ClockSampler(torch.cuda.current_device()) if (headline and tag == "fp64") else None
        ms, infos = timed_solves(solver, b, x, steps, args.tol, stream, dist, maxit)
        if clocks is not None:
            clk = clocks.stop()
        ms = dist.max(ms)
        rc, info = infos[-1]
        res[tag] = {"ms": ms, "rc": rc, "info": info, "x": x.clone(),
                    "shapes": shape_string(solver.info()[1])}
        # per-kernel records (every launch bracketed by events; host-driven loop)
        solver.profile(1)
        x.zero_()
        solver.solve(b, x, tol=args.tol, maxit=maxit)
        prof = solver.profile_read()
        # graph-part timings: CG part, V-cycle part, V-cycle from each level
        solver.profile(2)
        x.zero_()
        solver.solve(b, x, tol=args.tol, maxit=maxit)
        graph = {d["name"]: d["total_ms"] / max(1, d["launches"]) for d in solver.profile_read()}
        solver.profile(0)
        res[tag]["prof"] = prof
        res[tag]["graph"] = graph
        kern[tag] = {"kernels": prof, "graph_parts_ms": graph}
    solver.set_precision(amg.AMG_FP64)
    x64, x32 = res["fp64"]["x"], res["fp32"]["x"]
    err32 = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
    i64, i32 = res["fp64"]["info"], res["fp32"]["info"]
    n = p.n
    vc = {"fp64": vcycle_gbs(res["fp64"]["graph"], summary["vcycle_bytes_fp64"], 40.0 * n),
          "fp32": vcycle_gbs(res["fp32"]["graph"], summary["vcycle_bytes_fp32"], 80.0 * n)}
    kern["summary"] = summary
    kern["levels"] = levels
    kern["shapes"] = {"fp64": res["fp64"]["shapes"], "fp32": res["fp32"]["shapes"]}

    rec = {
        "fp64": {"ms": res["fp64"]["ms"], "iterations": i64["iterations"],
                 "true_rel_residual": i64["true_rel_residual"], "status": res["fp64"]["rc"]},
        "fp32_in_fp64": {"ms": res["fp32"]["ms"], "iterations": i32["iterations"],
                         "true_rel_residual": i32["true_rel_residual"], "status": res["fp32"]["rc"],
                         "rel_diff_vs_fp64_solution": err32,
                         "speedup_vs_fp64": res["fp64"]["ms"] / res["fp32"]["ms"]},
        "vcycle": vc,
        "shapes": {"fp64": res["fp64"]["shapes"], "fp32": res["fp32"]["shapes"]},
        "setup": {"total_ms": summary["total_setup_ms"], "host_ms": summary["host_setup_ms"],
                  "aggregation_ms": summary["aggregation_ms"],
                  "gpu_galerkin_ms": summary["gpu_galerkin_ms"], "gpu_other_ms": summary["gpu_other_ms"],
                  "levels": summary["num_levels"], "coarsest_n": summary["coarsest_n"],
                  "operator_complexity": summary["operator_complexity"],
                  "problem_generation_s": gen_s},
    }

    if headline:
        prof64 = res["fp64"]["prof"]
        top = max(prof64, key=lambda d: d["total_ms"])
        per_ms = top["total_ms"] / top["launches"]
        per_b = top["bytes"] / top["launches"]
        ach = per_b / (per_ms * 1e-3) / 1e9
        rec["roofline"] = {"bound": "hbm", "kernel": top["name"], "achieved": ach, "peak": peak,
                           "unit": "GB/s", "frac": ach / peak, "peak_source": peak_src,
                           "bytes_per_launch": per_b, "ms_per_launch": per_ms,
                           "share_of_solve": top["total_ms"] / sum(d["total_ms"] for d in prof64),
                           "traffic": kernel_traffic(top["name"], workload)}
        # kernels in the timed region: the profiled solve's launches (host-driven
        # loop) plus one loop-condition kernel per iteration of the device loop
        launches = sum(d["launches"] for d in prof64 if d["name"] != "zero")
        if i64.get("device_loop"):
            launches += i64["iterations"]
        rec["gpu_launches"] = launches * steps
        rec["clocks"] = clk
        rec["device_loop"] = i64.get("device_loop")
        if not args.no_e2e:
            bh = torch.from_numpy(p.b).pin_memory()
            xh = torch.zeros(p.n, dtype=torch.float64).pin_memory()
            bh_np, xh_np = bh.numpy(), xh.numpy()
            solver.solve_host(bh_np, xh_np, tol=args.tol, maxit=maxit, zero_guess=True)
            k = max(1, min(args.e2e_steps, steps))
            dist.barrier()
            t0 = time.perf_counter()
            for _ in range(k):
                solver.solve_host(bh_np, xh_np, tol=args.tol, maxit=maxit, zero_guess=True)
            e2e_ms = dist.max((time.perf_counter() - t0) * 1e3 / k)
            rec["e2e"] = {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 8 * p.n,
                          "d2h_bytes_per_step": 8 * p.n, "steps": k, "initial_guess": "zero",
                          "api": "amg_pcg_solve_host_zero_guess, pinned host buffers"}
            del bh, xh
    solver.close()
    del b, x, res
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec, kern, p


def gpu_time_on(args, p, dist):
    """FP64 time to tolerance of our solver on problem p (hierarchy resident),
    for a same-size comparison with the oracle sample."""
    import torch
    stream = torch.cuda.current_stream()
    solver = new_solver(args, p, stream)
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros_like(b)
    for _ in range(3):
        x.zero_()
        solver.solve(b, x, tol=args.tol, maxit=1000)
    ms, infos = timed_solves(solver, b, x, 5, args.tol, stream, dist, 1000)
    solver.close()
    return ms, infos[-1][1]["iterations"]


def run_ours(args, dist: Dist):
    import torch

    dev = dist.local_rank if dist.world > 1 else 0
    torch.cuda.set_device(dev)
    rec, kern, _ = measure_workload(args, dist, args.workload, args.grid, args.steps, args.warmup,
                                    True, args.kernels_out)
    all_kern = {args.workload: kern}
    others = {}
    for w in args.others:
        if w == args.workload:
            continue
        g = WORKLOADS[w][1]
        o, k2, _ = measure_workload(args, dist, w, g, args.steps, args.warmup, False, None)
        all_kern[w] = k2
        others[w] = {"fp64_ms": o["fp64"]["ms"], "fp64_iterations": o["fp64"]["iterations"],
                     "fp32_in_fp64_ms": o["fp32_in_fp64"]["ms"],
                     "fp32_in_fp64_iterations": o["fp32_in_fp64"]["iterations"],
                     "fp32_speedup": o["fp32_in_fp64"]["speedup_vs_fp64"],
                     "fp32_rel_diff_vs_fp64": o["fp32_in_fp64"]["rel_diff_vs_fp64_solution"],
                     "vcycle_fp64_frac": (o["vcycle"]["fp64"] or {}).get("frac_measured"),
                     "vcycle_fp32_frac": (o["vcycle"]["fp32"] or {}).get("frac_measured"),
                     "levels": o["setup"]["levels"]}

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1) -------------
    cpu = None
    cpu_omp = None
    if dist.world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(args.workload, args.cpu_grid, args.tol, 1, 0, min_seconds=10.0)
        gpu_ms, gpu_it = gpu_time_on(args, smp["problem"], dist)
        cpu = {"value": smp["solve_s"] * 1e3, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle PCG solve on the {args.cpu_grid}^3 instance of the workload "
                         f"({smp['n']} unknowns, {smp['iterations']} iterations, {smp['solves']} "
                         f"solves), unscaled; at its setup rate the {args.grid}^3 system would "
                         f"need about {smp['setup_s'] / smp['n'] * args.grid ** 3 / 60:.0f} min of "
                         f"oracle setup",
               "setup_s": smp["setup_s"], "cpu": cpu_model(), "host_cpu_count": os.cpu_count(),
               "gpu_fp64_ms_same_sample": gpu_ms, "gpu_iterations_same_sample": gpu_it}
        from oracle import oracle as O
        threads = O.threads(os.cpu_count() or 1)
        so = oracle_sample(args.workload, args.cpu_grid, args.tol, 1, 0, min_seconds=5.0, openmp=True)
        cpu_omp = {"value": so["solve_s"] * 1e3, "unit": UNIT, "cores": threads,
                   "kind": "oracle (OpenMP build of the same source)",
                   "setup_s": so["setup_s"], "iterations": so["iterations"]}

    # ---- a bounded serving leg (rank 0, N = 1) ------------------------------------
    serving = None
    if dist.world == 1 and args.serving_requests > 0:
        leg = serving_leg(args, args.serving_requests, agg_tile=4096)
        serving = {k: leg[k] for k in ("requests", "ok", "p50_ms", "p99_ms", "solves_per_s",
                                       "saturated_solves_per_s", "requests_per_batched_vcycle")}
        serving["median_setup_ms"] = leg["median_ms"]["setup_ms"]
        serving["median_solve_ms"] = leg["median_ms"]["solve_ms"]
        serving["workload"] = ("independent 3D 7-point solves, box sides U{16..96}, log-normal K "
                               "variance U[1,6]; FP32-in-FP64 to %g, Poisson arrivals at %.1f x "
                               "the saturated rate, host-tiled aggregation (4096 rows)"
                               % (args.tol, args.load))

    kpath = None
    if args.kernels_out and dist.rank == 0:
        try:
            os.makedirs(os.path.dirname(os.path.abspath(args.kernels_out)), exist_ok=True)
            with open(args.kernels_out, "w") as f:
                json.dump(all_kern, f)
            kpath = args.kernels_out
        except OSError:
            kpath = None

    line = {
        "metric": METRIC, "value": rec["fp64"]["ms"], "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["fp64"]["ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, args.workload, args.grid, dist.world),
                       launch_overlap=args.launch_overlap, coarsest_fp32=args.coarsest_fp32,
                       autotune=args.autotune,
                       device_loop=1 if args.device_loop is None else args.device_loop),
        "gpu_launches": rec["gpu_launches"],
        "e2e": rec.get("e2e"),
        "clocks": rec["clocks"],
        "cpu_baseline": cpu,
        "cpu_baseline_openmp": cpu_omp,
        "kernels_file": kpath,
        "setup": rec["setup"],
        "other_workloads": others,
        "serving": serving,
        "roofline": rec["roofline"],
        "device_loop": rec["device_loop"],
        "iterations": rec["fp64"]["iterations"],
        "true_rel_residual": rec["fp64"]["true_rel_residual"],
        "status": {"fp64": rec["fp64"]["status"], "fp32_in_fp64": rec["fp32_in_fp64"]["status"]},
        "vcycle": rec["vcycle"],
        "shapes": rec["shapes"],
        "fp32_in_fp64": rec["fp32_in_fp64"],
    }
    if dist.rank == 0:
        print(json.dumps(r4(line)), flush=True)


def profile_run(args):
    """One capped solve of the workload, for ncu captures of single kernels."""
    import torch
    from paper_1209_0960_gb300 import amg
    torch.cuda.set_device(0)
    p = make_problem(args.workload, args.grid)
    prec = amg.AMG_FP32_IN_FP64 if args.profile_fp32 else amg.AMG_FP64
    solver = amg.AMG(p.row_ptr, p.col, p.val, dim=3, launch_overlap=args.launch_overlap,
                     precision=prec, autotune=args.autotune, coarsest_fp32=args.coarsest_fp32,
                     device_loop=1 if args.device_loop is None else args.device_loop,
                     **({"coarsen_target": args.coarsen_target} if args.coarsen_target else {}))
    apply_lanes(solver, args)
    b = torch.from_numpy(p.b).cuda()
    x, rc, info = solver.solve(b, tol=args.tol, maxit=args.profile_run)
    torch.cuda.synchronize()
    print(f"profile run: rc {rc}, {info['iterations']} iterations")
    solver.close()


def _gen_request(k: int):
    from paper_1209_0960_gb300 import problems
    p = problems.serving_request(k)
    return k, p.row_ptr, p.col, p.val, p.b


def serving_leg(args, n_req, agg_tile=None):
    """Continuous-batching serving on the current GPU: FP32-in-FP64 AMG-PCG to
    --tol for n_req independent requests.  Phase 1 submits a burst to measure
    the saturated rate; phase 2 replays all requests with Poisson arrivals at
    --load times that rate and records latency percentiles.  The requests are
    generated in spawned processes."""
    import multiprocessing as mp
    import numpy as np
    import torch
    from paper_1209_0960_gb300 import amg
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        reqs = sorted(pool.map(_gen_request, range(n_req), chunksize=8), key=lambda t: t[0])
    threads = args.setup_threads or max(1, (os.cpu_count() or 4) - 3)
    tile = args.aggregation_tile if agg_tile is None else agg_tile
    srv = amg.Server(dim=3, max_slots=args.slots, setup_threads=threads,
                     aggregation_tile=tile, aggregation_device=args.aggregation_device,
                     autotune=args.autotune, host_threads=args.host_threads,
                     batch_vcycles=args.batch_vcycles,
                     **({"device_loop": args.device_loop} if args.device_loop is not None else {}))

    def drain(tickets, results):
        while len(results) < len(tickets):
            for t in tickets:
                if t not in results:
                    r = srv.poll(t)
                    if r is not None:
                        results[t] = r
            time.sleep(0.0005)

    # phase 1: saturated throughput on a burst (also warms the pinned pool)
    burst = reqs[:max(1, min(n_req, 4 * args.slots))]
    t0 = time.perf_counter()
    tk = [srv.submit(rp, ci, va, b, args.tol) for _, rp, ci, va, b in burst]
    res = {}
    drain(tk, res)
    sat_rate = len(burst) / (time.perf_counter() - t0)

    # phase 2: Poisson arrivals
    rate = args.rate if args.rate > 0 else args.load * sat_rate
    rng = np.random.default_rng(1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    res2, pending = {}, []
    t0 = time.perf_counter()
    i = 0
    while i < n_req or pending:
        now = time.perf_counter() - t0
        while i < n_req and arrivals[i] <= now:
            _, rp, ci, va, b = reqs[i]
            pending.append(srv.submit(rp, ci, va, b, args.tol))
            i += 1
        still = []
        for t in pending:
            r = srv.poll(t)
            if r is None:
                still.append(t)
            else:
                res2[t] = r
        pending = still
        time.sleep(0.0002)
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array([r[3]["total_ms"] for r in res2.values()])
    sizes = [reqs[k][1].shape[0] - 1 for k in range(n_req)]
    return {
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "solves_per_s": n_req / wall, "saturated_solves_per_s": sat_rate, "offered_rate_per_s": rate,
        "requests": n_req, "ok": sum(1 for r in res2.values() if r[0] == amg.AMG_OK),
        "worst_true_rel_residual": max(r[2]["true_rel_residual"] for r in res2.values()),
        "median_ms": {k: float(np.median([r[3][k] for r in res2.values()]))
                      for k in ("queue_ms", "setup_ms", "solve_ms")},
        "peak_in_flight": stats["peak_running"], "slots": args.slots, "setup_threads": threads,
        "aggregation_tile": tile, "batch_vcycles": args.batch_vcycles,
        "batched_vcycles": stats["batched_vcycles"],
        "requests_per_batched_vcycle": (stats["batched_requests"] / stats["batched_vcycles"]
                                        if stats["batched_vcycles"] else 0.0),
        "device_loop": srv.params.params.device_loop,
        "unknowns": {"min": int(min(sizes)), "median": int(np.median(sizes)), "max": int(max(sizes))},
    }


def run_serving(args):
    """The serving workload alone, with its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    leg = serving_leg(args, args.serving)
    line = {
        "metric": "serving: p50/p99 request latency (submit to solution on the host) and solves/s",
        "value": leg["p50_ms"], "unit": "ms", "higher_is_better": False,
        **{k: v for k, v in leg.items() if k != "p50_ms"},
        "autotune": args.autotune, "host_threads": args.host_threads,
        "aggregation_device": args.aggregation_device,
        "dtype": "f32 V-cycle in f64 CG", "data": "synthetic",
        "config": {"workload": "serving stream: independent 3D 7-point FV solves, box sides "
                               "U{16..96}, log-normal K variance U[1,6], correlation length 0.1, "
                               "Poisson arrivals; FP32-in-FP64 AMG-PCG to %g" % args.tol,
                   "load": args.load},
    }
    print(json.dumps(r4(line)), flush=True)


def main():
    args = parse_args()
    if args.profile_run > 0:
        profile_run(args)
        return
    if args.serving > 0:
        run_serving(args)
        return
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
