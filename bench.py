#!/usr/bin/env python
"""Benchmark of the sparsified-AMG PCG solver on GB300.

Workload (`poisson3d7`, the default): 3D 7-point Poisson on a 128^3 grid
(n = 2,097,152, nnz = 14,581,760), right-hand side uniform[-1, 1) from seed 1,
x0 = 0.  One step = the whole hot path on inputs already resident in HBM:
GPU setup (strength, PMIS, direct interpolation, Galerkin SpGEMM), Sparse
Galerkin sparsification with diagonal lumping at gamma = 0.1 on levels >= 1,
ell1 diagonals, coarse Cholesky, then PCG with one V(1,1) per iteration to
||b - A x|| / ||b|| <= 1e-8, FP64.  value = solves per second over all ranks.

Also reported, all outside the timed region:
  * the roofline of the dominant solve-phase kernel (algorithmic bytes /
    CUDA-event time vs the measured HBM peak, and the FP64 pipe);
  * the same metric end to end through the C ABI with host buffers;
  * `arms`: solve-only time to 1e-8 (setup excluded, median of 5) for the
    Galerkin, gamma in {0.01, 0.1, 1} and adaptive hierarchies of the same
    workload, each with an eager per-kernel breakdown of where the time goes;
  * `communication`: the paper's communication measure -- every level split
    into 8 and 64 row blocks (amg_partition), messages and ghost values per
    product for Galerkin and sparsified hierarchies, and the alpha-beta model
    time of a V-cycle's relaxation products (a model, not a GPU measurement);
  * `legs` (one GPU only): the metric's other configurations, each with its
    own config, CUDA-event timing and sampled clocks -- c3: 27-point 192^3
    FP64 vs FP32 vs FP32 + BF16 time to 1e-8; c4: lognormal FV 160^3 batched
    solves/s for k in {1, 8, 32, 64} against FP64 single solves; c5: serving
    8 resident hierarchies under Poisson arrivals at 200/s (p50 / p99, solves/s);
  * `cpu_baseline`: the CPU oracle on every host core (its all-core build:
    the solve phase's loops under OpenMP, setup sequential), with the
    sequential build's figure beside it.
`--impl reference` times the all-core CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os

# before any CUDA context exists: one hardware queue per stream (the serving
# workload runs eight hierarchies and a copy stream side by side)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 solve & V-cycle HBM GB/s, sparse vs Galerkin; serving p99"
UNIT = "solves/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--gamma", type=float, default=0.1)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--no-arms", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-legs", action="store_true",
                   help="skip the c3 / c4 / c5 legs of the default line (27-point precision arms, batched "
                        "lognormal, serving)")
    p.add_argument("--leg-serve-seconds", type=float, default=12.0,
                   help="arrival window of the serving leg in the default line")
    p.add_argument("--workload", default="poisson3d7",
                   choices=["poisson3d7", "poisson3d27", "lognormal-batched", "serving", "lump", "aniso"],
                   help="poisson3d7 (default, the bench line): 3D 7-pt 128^3; poisson3d27: 27-pt 192^3 "
                        "precision arms; lognormal-batched: lognormal FV 160^3 batched k in {1,8,32,64}; "
                        "serving: 8 resident hierarchies, Poisson arrivals at 200/s; "
                        "lump: 3D 7-pt 128^3, diagonal vs full lumping, CG vs GMRES; "
                        "aniso: rotated anisotropic Q1 2D 2048^2 (theta pi/8, eps 1e-3), GMRES arms "
                        "(Galerkin, Sparse, Hybrid, non-Galerkin)")
    p.add_argument("--serve-seconds", type=float, default=20.0)
    p.add_argument("--serve-batch", type=int, default=8,
                   help="serving: column slots per hierarchy (the server's max_batch); 8 measured best for the "
                        "200/s stream over 8 hierarchies (p99 272 ms against 462 at 16 and 938 at 32)")
    p.add_argument("--batch-k", type=int, nargs="*", default=None,
                   help="lognormal-batched: the widths to run (default 1 8 32 64)")
    p.add_argument("--lump", default="diag", choices=["diag", "strong"],
                   help="sparsify: diagonal lumping (Algorithm 3b, default) or full lumping to strong neighbours "
                        "(Algorithm 3)")
    p.add_argument("--krylov", default="cg", choices=["cg", "gmres"],
                   help="outer solver: PCG (default) or restarted GMRES(30)")
    p.add_argument("--eager", action="store_true",
                   help="launch the PCG iterations one kernel at a time (no CUDA graph; for ncu launch lists)")
    p.add_argument("--ncu-setup", action="store_true",
                   help="profiling aid: one warm-up setup, then one setup between cudaProfilerStart/Stop")
    p.add_argument("--ncu-solve", action="store_true",
                   help="set up once, then run one solve between cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return p.parse_args()


def workload_config(args):
    n = args.grid ** 3
    lump = "full lumping to strong neighbours (Algorithm 3)" if args.lump == "strong" else \
        "diagonal lumping (Algorithm 3b)"
    solver = "GMRES(30)" if args.krylov == "gmres" else "PCG"
    return {
        "workload": f"3D 7-point Poisson {args.grid}^3 (n={n}), Sparse Galerkin gamma={args.gamma} on levels>=1, "
                    f"{lump}, {solver} + V(1,1) l1-Jacobi to {args.tol:g}, FP64; step = GPU setup + sparsify + solve",
        "grid": args.grid, "n": n, "gamma": args.gamma, "tol": args.tol, "precision": "fp64",
        "lump": args.lump, "krylov": args.krylov,
        "theta": 0.25, "coarsening": "PMIS", "interpolation": "direct",
        "l2_policy": "inputs larger than L2 (A = 175 MB FP64 CSR at 128^3)",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 pipe of a GB300: one FP64 warp instruction per 16 clocks per SM, i.e. 2 FMA per clock per SM
# (measured 2.00 with a DFMA throughput probe); peak = 2 x 152 SMs x the sampled SM clock.
FP64_FMA_PER_CLK_SM = 2.0
GB300_SMS = 152


def fp64_ops_per_launch(kind, level, n, nnz, precision):
    """FP64 lane operations (FMA / add / mul, one each) of one launch of a solve-phase kernel class,
    counted from the arithmetic each kernel performs per stored entry and per row."""
    if precision != "fp64" and kind not in ("pcg_Ap_dot", "pcg_vector"):
        return None
    if kind == "relax_pre_residual":
        return nnz + n                      # s = A x; r = b - s
    if kind == "relax_post":
        return nnz + (3 if level == 0 else 2) * n   # x + d (b - s); level 0 adds r.z (plain CG: no z.q)
    if kind == "pcg_Ap_dot":
        return nnz + n                      # q = A p; p.q
    if kind == "pcg_vector":
        return 4 * n                        # x += a p; r -= a q; x0 = d r; r.r
    return None


def ncu_traffic():
    """Per-launch DRAM bytes of kernels captured with ncu (profiles/)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            key, rows, nnz, b = line.split()[:4]
            out[key] = (int(rows), int(nnz), float(b))
    return out


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def oracle_step(A, b, gamma, tol, lump="diag", krylov="cg", omp=False):
    """One oracle step (setup + sparsify + solve); returns (total s, info,
    {"setup_s", "solve_s"}).  omp: the all-core timing build."""
    import oracle

    t0 = time.perf_counter()
    h = oracle.Hierarchy(A, omp=omp)
    h.sparsify([0.0, gamma], lump=1 if lump == "strong" else 0)
    t1 = time.perf_counter()
    x, info = h.gmres(b, tol=tol) if krylov == "gmres" else h.pcg(b, tol=tol)
    t2 = time.perf_counter()
    assert info.status == 0, info
    return t2 - t0, info, {"setup_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import amg_inputs as gen
    import oracle

    oracle.build(omp=True)
    cores = host_cores()
    A = gen.poisson3d_7pt(args.grid)
    b = gen.rhs_uniform(A.n, 1)
    budget = 200.0 / max(1, args.steps + args.warmup)  # seconds per step
    # one untimed full-size step sizes the sample: full size if it fits the
    # per-step budget, else the largest sub-grid that does (value scaled by n)
    t_full, _, _ = oracle_step(A, b, args.gamma, args.tol, args.lump, args.krylov, omp=True)
    N, As, bs, scale = args.grid, A, b, 1.0
    if t_full > budget:
        N = max(16, int(args.grid * (budget / t_full) ** (1.0 / 3.0)))
        As = gen.poisson3d_7pt(N)
        bs = gen.rhs_uniform(As.n, 1)
        scale = As.n / A.n
    for _ in range(max(0, args.warmup - (1 if scale == 1.0 else 0))):
        oracle_step(As, bs, args.gamma, args.tol, args.lump, args.krylov, omp=True)
    times = []
    its = None
    for _ in range(args.steps):
        dt, info, _ = oracle_step(As, bs, args.gamma, args.tol, args.lump, args.krylov, omp=True)
        times.append(dt)
        its = info.iterations
    total = sum(times)
    value = args.steps / total * scale
    where = (f"full workload ({args.grid}^3) per step" if scale == 1.0 else
             f"{N}^3 sub-grid per step (n={As.n}), value scaled by n ratio {scale:.4f} (AMG cost is O(n))")
    sample = (f"{where}; oracle all-core build: setup and sparsify sequential, PCG's SpMV, vector and dot loops "
              f"on {cores} OpenMP threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args), "iterations": its,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline_leg(args, A, b):
    """The oracle on this host's cores: the all-core build (timed baseline)
    and the sequential parity build, one full step each on the full workload."""
    import oracle

    oracle.build(omp=True)
    cores = host_cores()
    dt, info, ph = oracle_step(A, b, args.gamma, args.tol, args.lump, args.krylov, omp=True)
    dt1, info1, ph1 = oracle_step(A, b, args.gamma, args.tol, args.lump, args.krylov, omp=False)
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": (f"one full step at {args.grid}^3 ({info.iterations} its): oracle all-core build, setup and "
                       f"sparsify sequential, PCG's SpMV, vector and dot loops on {cores} OpenMP threads"),
            "phases_s": ph,
            "single_thread": {"value": 1.0 / dt1, "cores": 1, "phases_s": ph1, "iterations": info1.iterations}}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
KIND_NAMES = {0: "relax_pre_residual", 1: "restrict", 2: "prolong", 3: "relax_post", 4: "coarse_solve",
              5: "pcg_Ap_dot", 6: "pcg_vector"}  # under GMRES: 5 = A z, 6 = orthogonalisation and updates
SETUP_KIND_NAMES = {8: "strength", 9: "cf_split", 10: "interpolation", 11: "galerkin_spgemm",
                    12: "level_maps_minimal_pattern", 13: "sparsify", 14: "cycle_prep", 15: "coarse_cholesky"}


def aggregate_replicas(elapsed_s: float, steps: int, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank did `steps`
    solves; the job took the slowest rank's time (max over ranks)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch

        world = dist.get_world_size()
        t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return world * steps / elapsed_s, elapsed_s, world


def collect_timing(h, nlev):
    rows = []
    for kind in range(7):
        for l in range(nlev):
            n, ms, by = h.timing_get(kind, l)
            if n:
                rows.append({"kind": KIND_NAMES[kind], "level": l, "launches": n, "ms": ms, "bytes": by})
    return rows


def _median_phases(runs):
    if not runs:
        return None
    out = {}
    for k in runs[0]:
        if k.endswith("_by_level"):
            out[k] = [round(statistics.median(r[k][i] for r in runs), 3) for i in range(len(runs[0][k]))]
        else:
            out[k] = round(statistics.median(r[k] for r in runs), 3)
    return out


def collect_setup_timing(h, nlev):
    """Setup phase -> milliseconds summed over levels (event spans on the setup stream),
    plus the same per level under "<phase>_by_level"."""
    out = {}
    for kind, name in SETUP_KIND_NAMES.items():
        per = [h.timing_get(kind, l)[1] for l in range(nlev)]
        out[name] = round(sum(per), 3)
        out[name + "_by_level"] = [round(x, 3) for x in per]
    return out


# ---------------------------------------------------------------------------
# other workloads (measured one line each; not the default bench line)
# ---------------------------------------------------------------------------
def _events_ms(fn, reps=3):
    import torch

    times, out = [], None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), out


def leg_c3(args, reps=3):
    """27-point 192^3: FP64 vs FP32 vs FP32+BF16 cycles on the Galerkin and the
    gamma = 0.1 hierarchies.  Time to 1e-8 = the solve (setup excluded; median
    of `reps`, CUDA events on the current stream); the error of each solution
    is stated against the FP64 solve of the same hierarchy and against the FP64
    Galerkin one."""
    import torch

    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    N = 192 if args.grid == 128 else args.grid
    A = gen.poisson3d_27pt(N)
    b = gen.rhs_uniform(A.n, 1)
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
    A_dev = amg.amg.csr_struct(rp, ci, va)
    bd = torch.from_numpy(b).cuda()
    res, xgal = {}, None
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for g in (0.0, 0.1):
        x64 = None
        for prec, pname in ((0, "fp64"), (1, "fp32"), (2, "fp32_bf16")):
            setup_ms, hs = _events_ms(lambda: amg.Hierarchy.setup(A_dev, gamma=[0.0, g] if g else None,
                                                                  precision=prec), reps=1)
            h = hs
            xd = torch.zeros_like(bd)
            ms, (x, info) = _events_ms(lambda: h.solve(bd, xd, tol=args.tol), reps=reps)
            if prec == 0:
                x64 = x.clone()
                if g == 0.0:
                    xgal = x.clone()
            res[f"gamma{g}_{pname}"] = {
                "time_to_tol_ms": round(ms, 3), "setup_ms": round(setup_ms, 3), "iterations": info.iterations,
                "status": info.status, "final_relres": info.final_relres,
                "rel_err_vs_fp64_same_hierarchy": float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64)),
                "rel_err_vs_fp64_galerkin": float(torch.linalg.norm(x - xgal) / torch.linalg.norm(xgal)),
                "levels": h.num_levels,
                "nnz_per_level": [h.level_stats(l)["nnz_operator"] for l in range(h.num_levels)],
                "value_bytes": [h.level_stats(l)["value_bytes"] for l in range(h.num_levels)]}
            del h, hs, x
    clocks = sampler.stop()
    best = min(res, key=lambda k: res[k]["time_to_tol_ms"])
    return {"config": {"workload": f"3D 27-point Poisson {N}^3 (n={A.n}, nnz={A.nnz}), RHS seed 1, tol {args.tol:g}",
                       "arms": "Galerkin and gamma 0.1 x {FP64, FP32 cycle, FP32 cycle + BF16 values on levels >= 2}; "
                               "outer PCG / flexible CG in FP64",
                       "timing": f"solve only, median of {reps}, CUDA events"},
            "unit": "ms", "arms": res, "fastest": best,
            "speedup_fp32_bf16_vs_fp64_gamma0.1": round(res["gamma0.1_fp64"]["time_to_tol_ms"] /
                                                        res["gamma0.1_fp32_bf16"]["time_to_tol_ms"], 3),
            "clocks": clocks}


def run_poisson3d27(args):
    print(json.dumps(leg_c3(args)))


def leg_c4(args, reps=3):
    """Lognormal FV 160^3, gamma 0.1: FP64 single solves against the FP32-cycle
    batched solves for k in {1, 8, 32, 64} (solves/s; median of `reps`)."""
    import numpy as np
    import torch

    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    N = 160 if args.grid == 128 else args.grid
    A = gen.fv7_lognormal(N, seed=3)
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
    A_dev = amg.amg.csr_struct(rp, ci, va)
    out = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    h64 = amg.Hierarchy.setup(A_dev, gamma=[0.0, 0.1], precision=0)
    b0 = torch.from_numpy(gen.rhs_uniform(A.n, 0)).cuda()
    ms64, (_, i64) = _events_ms(lambda: h64.solve(b0, tol=args.tol), reps=reps)
    out["fp64_single"] = {"ms": round(ms64, 3), "solves_per_s": round(1e3 / ms64, 2), "iterations": i64.iterations}
    del h64
    h = amg.Hierarchy.setup(A_dev, gamma=[0.0, 0.1], precision=1)
    for k in args.batch_k or (1, 8, 32, 64):
        B = torch.from_numpy(np.stack([gen.rhs_uniform(A.n, c) for c in range(k)], axis=1)).cuda().contiguous()
        if k == 1:
            bb = B[:, 0].contiguous()
            ms, (_, inf) = _events_ms(lambda: h.solve(bb, tol=args.tol), reps=reps)
            its, ok = [inf.iterations], inf.status == 0 and inf.final_relres <= args.tol
        else:
            ms, (_, infos) = _events_ms(lambda: h.solve_batch(B, tol=args.tol), reps=reps)
            its = [i.iterations for i in infos]
            ok = all(i.status == 0 and i.final_relres <= args.tol for i in infos)
        out[f"fp32_k{k}"] = {"ms": round(ms, 3), "solves_per_s": round(k * 1e3 / ms, 2), "iterations_max": max(its),
                             "iterations_min": min(its), "all_converged": ok}
        del B
    clocks = sampler.stop()
    best = max((v["solves_per_s"], k) for k, v in out.items())
    return {"config": {"workload": f"lognormal FV 7-point {N}^3 (n={A.n}, sigma 2, seed 3), gamma 0.1, tol {args.tol:g}",
                       "arms": "FP64 single solve vs FP32 cycle / FP64 outer CG, batched k RHS (seeds 0..k-1)",
                       "timing": f"median of {reps}, CUDA events, setup excluded"},
            "unit": "solves/s", "arms": out, "best": best[1],
            "speedup_best_vs_fp64_single": round(best[0] / out["fp64_single"]["solves_per_s"], 3),
            "clocks": clocks}


def run_lognormal_batched(args):
    print(json.dumps(leg_c4(args)))


def leg_c5(args, seconds=None):
    """Serving: 8 resident hierarchies, Poisson arrivals at 200/s, continuous batching.

    The right-hand sides are generated before the clock starts (a pool of
    seeded vectors per hierarchy, used in turn), and a waiter thread retires
    tickets while requests keep arriving, so the client does not limit the
    offered rate; the line reports the rate it achieved and its worst lag
    behind the arrival schedule."""
    import queue
    import threading

    import numpy as np

    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    kinds = [("2d5", 256), ("2d5", 512), ("2d5", 1024), ("2d5", 2048),
             ("3d7", 32), ("3d7", 64), ("3d7", 96), ("3d7", 128)]
    hs, ns = [], []
    for kind, N in kinds:
        A = gen.generate(kind, N)
        hs.append(amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1))
        ns.append(A.n)
    pool_per_h = 4
    pool = [[gen.rhs_uniform(ns[hid], 10_000 + pool_per_h * hid + k) for k in range(pool_per_h)]
            for hid in range(len(hs))]
    srv = amg.Server(max_batch=args.serve_batch)
    ids = [srv.register(h) for h in hs]
    rng = np.random.default_rng(5)
    rate, T = 200.0, seconds or args.serve_seconds
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * T * 1.5)))
    arrivals = arrivals[arrivals < T]
    picks = rng.integers(0, len(hs), size=len(arrivals))

    pending: queue.Queue = queue.Queue()
    results = []

    def waiter():
        while True:
            item = pending.get()
            if item is None:
                return
            t, hid = item
            st, _, info = srv.wait(t, ids[hid], timeout_ms=600000)
            results.append((st, info))

    th = threading.Thread(target=waiter)
    th.start()
    lag = 0.0
    import torch

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0 = time.perf_counter()
    for r, (ta, hid) in enumerate(zip(arrivals, picks)):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        else:
            lag = max(lag, now - ta)
        pending.put((srv.submit(ids[hid], pool[hid][r % pool_per_h]), hid))
    t_sub = time.perf_counter() - t0
    pending.put(None)
    th.join()
    wall = time.perf_counter() - t0
    srv.close()
    clocks = sampler.stop()
    bad = sum(1 for st, info in results if st != 0 or info.final_relres > args.tol)
    lat = np.array([info.solve_ms for _, info in results])
    its = [info.iterations for _, info in results]
    return {"config": {"workload": "serving 8 resident hierarchies (2D 256^2, 512^2, 1024^2, 2048^2; 3D 32^3, 64^3, "
                                   "96^3, 128^3; gamma 0.1, FP32 cycle, FP64 outer CG), uniform hierarchy choice, "
                                   f"Poisson arrivals at {rate:g}/s for {T:g} s, tol {args.tol:g}, max_batch {args.serve_batch}",
                       "timing": "latency = submit to result per request (host clock); solves/s over the wall time "
                                 "from the first arrival to the last result"},
            "requests": len(results), "failed": bad, "solves_per_s": round(len(results) / wall, 2),
            "offered_per_s": round(len(results) / T, 2), "submitted_per_s": round(len(results) / t_sub, 2),
            "client_max_lag_ms": round(1e3 * lag, 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_ms": round(float(lat.max()), 3), "iterations_median": float(np.median(its)), "clocks": clocks}


def run_serving(args):
    print(json.dumps(leg_c5(args)))


def _lumping_arms(args, A, arms, workload):
    """One line of arms: setup (median of 3, events), the sparsify phase
    (setup_timing), solve (median of 3), iterations and operator sizes."""
    import torch

    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    b = gen.rhs_uniform(A.n, 1)
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
    A_dev = amg.amg.csr_struct(rp, ci, va)
    bd = torch.from_numpy(b).cuda()
    out = {}
    for name, opts in arms:
        hs = []  # every timed hierarchy is kept until the timing ends (no teardown inside it)
        try:
            ms_setup, _ = _events_ms(lambda: hs.append(amg.Hierarchy.setup(A_dev, **opts)))
        except amg.AmgError as e:  # e.g. a non-Galerkin operator losing its positive diagonal
            out[name] = {"setup_status": e.status, "setup_error": str(e)}
            continue
        del hs
        ht = amg.Hierarchy.setup(A_dev, setup_timing=1, **opts)
        phases = collect_setup_timing(ht, ht.num_levels)
        del ht
        h = amg.Hierarchy.setup(A_dev, **opts)
        xd = torch.zeros_like(bd)
        ms_solve, (x, info) = _events_ms(lambda: h.solve(bd, xd, tol=args.tol, max_it=1000))
        nnz = [h.level_stats(l)["nnz_operator"] for l in range(h.num_levels)]
        gal = [h.level_stats(l)["nnz_galerkin"] for l in range(h.num_levels)]
        out[name] = {"setup_ms": round(ms_setup, 3), "sparsify_ms": phases.get("sparsify"),
                     "solve_ms": round(ms_solve, 3), "iterations": info.iterations, "status": info.status,
                     "final_relres": info.final_relres,
                     "ms_per_iteration": round(ms_solve / max(info.iterations, 1), 4),
                     "conv_factor": round(info.conv_factor, 4),
                     "operator_complexity": round(sum(nnz) / nnz[0], 4),
                     "galerkin_complexity": round(sum(gal) / gal[0], 4), "nnz_per_level": nnz}
        del h
    print(json.dumps({"workload": workload, "unit": "ms", "tol": args.tol, "arms": out}))


def run_lump(args):
    """3D 7-point 128^3: Algorithm 3b (diagonal) vs Algorithm 3 (full lumping to
    strong neighbours), each under PCG and GMRES(30), gamma 0.1 and 1.0 on
    every coarse level."""
    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    A = gen.poisson3d_7pt(args.grid)
    arms = [("galerkin_cg", {})]
    for g in (0.1, 1.0):
        for lump, ln in ((amg.LUMP_DIAG, "diag"), (amg.LUMP_STRONG, "full")):
            for kr, kn in ((amg.KRYLOV_CG, "cg"), (amg.KRYLOV_GMRES, "gmres")):
                arms.append((f"{ln}_{kn}_gamma{g}", {"gamma": [0.0, g], "lump": lump, "krylov": kr}))
    # the paper's comparator: non-Galerkin (thinned inside the setup loop), GMRES
    for sched, sn in (([0.0, 0.1], "0.1"), ([0.0, 0.0, 1.0], "0-1"), ([0.0, 1.0], "1.0")):
        for lump, ln in ((amg.LUMP_DIAG, "diag"), (amg.LUMP_STRONG, "full")):
            arms.append((f"nongalerkin_{ln}_gmres_gamma{sn}", {"gamma": sched, "lump": lump,
                                                              "method": amg.METHOD_NONGALERKIN,
                                                              "krylov": amg.KRYLOV_GMRES}))
    _lumping_arms(args, A, arms, f"lump: 3D 7-point {args.grid}^3 (n={A.n}), Sparse Galerkin")


def run_aniso(args):
    """Rotated anisotropic diffusion (Q1, theta = pi/8, eps = 1e-3) on a 2D
    grid: Galerkin, Sparse, Hybrid and non-Galerkin with diagonal and full
    lumping, all under GMRES(30)."""
    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg

    N = 2048 if args.grid == 128 else args.grid
    A = gen.rotated_aniso_q1(N)
    G = amg.KRYLOV_GMRES
    arms = [("galerkin", {"krylov": G})]
    for sched, sn in (([0.0, 0.1, 1.0], "0.1-1"), ([0.0, 1.0], "1")):
        for method, mn in ((amg.METHOD_SPARSE, "sparse"), (amg.METHOD_HYBRID, "hybrid"),
                           (amg.METHOD_NONGALERKIN, "nongalerkin")):
            for lump, ln in ((amg.LUMP_DIAG, "diag"), (amg.LUMP_STRONG, "full")):
                arms.append((f"{mn}_{ln}_gamma{sn}", {"gamma": sched, "method": method, "lump": lump,
                                                       "krylov": G}))
    _lumping_arms(args, A, arms, f"aniso: rotated anisotropic Q1 {N}^2 (n={A.n}, theta pi/8, eps 1e-3), GMRES(30)")


# the paper's alpha-beta model (Section 4), with its Blue Waters constants
ALPHA_S, BETA_S_PER_BYTE = 1.8e-6, 1.8e-9


def communication(A_dev, parts_list=(8, 64)):
    """The paper's communication measure for the bench workload: each level
    split into row blocks (amg_partition), messages and ghost values per
    product of the relaxed operator (Galerkin vs sparsified), P and R, and
    the alpha-beta model time of one V(1,1) cycle on the busiest block
    (2 products with the relaxed operator, 1 with R, 1 with P per level).
    The model uses the paper's constants: a model of a distributed run, not
    a measurement on this GPU."""
    import paper_1512_04629_gb300 as amg

    out = {"model": f"alpha-beta (Section 4), alpha = {ALPHA_S:g} s, beta = {BETA_S_PER_BYTE:g} s/byte, 8-byte values",
           "by_parts": {}}
    for parts in parts_list:
        per = {}
        for name, g in (("galerkin", 0.0), ("gamma_0.1", 0.1), ("gamma_1.0", 1.0)):
            h = amg.Hierarchy.setup(A_dev, gamma=[0.0, g] if g else None)
            h.partition(parts)
            levels, model = [], 0.0
            for l in range(h.num_levels):
                st = h.comm_stats(l)
                levels.append({"messages": st["messages"], "halo_values": st["halo_values"],
                               "max_messages": st["max_messages"], "max_halo": st["max_halo"],
                               "messages_P": st["messages_p"], "halo_P": st["halo_p"],
                               "messages_R": st["messages_r"], "halo_R": st["halo_r"]})
                if l + 1 < h.num_levels:  # the coarsest level is a dense solve, not a product
                    model += 2 * (ALPHA_S * st["max_messages"] + BETA_S_PER_BYTE * 8 * st["max_halo"])
            per[name] = {"levels": levels, "model_us_per_vcycle_relaxation": round(1e6 * model, 2),
                         "messages_per_vcycle": 2 * sum(v["messages"] for v in levels[:-1]),
                         "halo_values_per_vcycle": 2 * sum(v["halo_values"] for v in levels[:-1])}
            del h
        out["by_parts"][str(parts)] = per
    return out


def setup_roofline(h, phases):
    """Throughput of the Galerkin products A P and R (A P) per level, from the
    exported operators: products (the multiply-adds of the row-by-row
    product, summed over both products) and algorithmic bytes (read A, P, R
    and A P once, write A P and A_c once; 4-byte indices, 8-byte values),
    against the measured Galerkin phase time of that level."""
    import numpy as np

    out, tot_p, tot_b, tot_ms = [], 0, 0.0, 0.0
    for l in range(h.num_levels - 1):
        A = h.export(l, "A").to_scipy()
        P = h.export(l, "P").to_scipy()
        Ac = h.export(l + 1, "A")
        AP = (A @ P).tocsr()
        AP.sort_indices()
        p_rows = np.diff(P.indptr)
        ap_rows = np.diff(AP.indptr)
        prod_ap = int(p_rows[A.indices].sum())  # every a_ik meets row k of P
        R = P.T.tocsr()
        prod_rap = int(ap_rows[R.indices].sum())  # every r_ci meets row i of A P
        nbytes = 12.0 * (A.nnz + 2 * P.nnz + 2 * AP.nnz + Ac.nnz) + 4.0 * (A.shape[0] + 2 * P.shape[0] + 2 * R.shape[0])
        ms = phases["galerkin_spgemm_by_level"][l]
        out.append({"level": l, "products": prod_ap + prod_rap, "nnz_AP": int(AP.nnz), "nnz_Ac": int(Ac.nnz),
                    "ms": ms, "Gproducts_per_s": round((prod_ap + prod_rap) / (ms * 1e-3) / 1e9, 3),
                    "GBps": round(nbytes / (ms * 1e-3) / 1e9, 1)})
        tot_p += prod_ap + prod_rap
        tot_b += nbytes
        tot_ms += ms
    return {"what": "Galerkin A P and R (A P): products and algorithmic bytes per measured phase time",
            "levels": out, "Gproducts_per_s": round(tot_p / (tot_ms * 1e-3) / 1e9, 3),
            "GBps": round(tot_b / (tot_ms * 1e-3) / 1e9, 1), "ms": round(tot_ms, 3)}


def solve_arms(args, A_dev, nnz0, bd, xd, stream, reps=5):
    """Solve-only time to tol (setup excluded) on the bench workload for the
    Galerkin, gamma in {0.01, 0.1, 1} and adaptive (Algorithm 5 from gamma 1)
    hierarchies: median of `reps` solves after one warm-up, CUDA events on the
    current stream.  The adaptive arm re-sparsifies to gamma 1 before every
    rep, outside the timed span.  One more rep per arm, eager with per-kernel
    event timing, attributes the time to V-cycle kernels, PCG kernels and (for
    the adaptive arm) the reintroductions' re-sparsification and cycle
    preparation."""
    import torch

    import paper_1512_04629_gb300 as amg

    arms = {}
    for name, g, adaptive in [("galerkin", 0.0, False), ("gamma_0.01", 0.01, False), ("gamma_0.1", 0.1, False),
                              ("gamma_1.0", 1.0, False), ("adaptive_from_1.0", 1.0, True)]:
        t0 = time.perf_counter()
        h = amg.Hierarchy.setup(A_dev, gamma=[0.0, g] if g > 0 else None)
        torch.cuda.synchronize()
        setup_ms = 1e3 * (time.perf_counter() - t0)
        sol, info = [], None
        for rep in range(reps + 1):
            if adaptive:
                h.sparsify([0.0, g])
                torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = h.solve(bd, xd, tol=args.tol, adaptive=adaptive)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                sol.append(e0.elapsed_time(e1))
        assert info.status == 0 and info.final_relres <= args.tol, info.as_dict()
        # attribution pass (eager: per-kernel events)
        if adaptive:
            h.sparsify([0.0, g])
        torch.cuda.synchronize()
        h.timing_reset()
        h.timing_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, tinfo = h.solve(bd, xd, tol=args.tol, adaptive=adaptive)
        e1.record(stream)
        torch.cuda.synchronize()
        h.timing_enable(False)
        eager_ms = e0.elapsed_time(e1)
        rows = collect_timing(h, h.num_levels)
        vms = sum(r["ms"] for r in rows if r["kind"] not in ("pcg_Ap_dot", "pcg_vector"))
        vby = sum(r["bytes"] for r in rows if r["kind"] not in ("pcg_Ap_dot", "pcg_vector"))
        pms = sum(r["ms"] for r in rows if r["kind"] in ("pcg_Ap_dot", "pcg_vector"))
        reint = sum(h.timing_get(kind, l)[1] for kind in (13, 14) for l in range(h.num_levels))
        oc = sum(h.level_stats(l)["nnz_operator"] for l in range(h.num_levels)) / nnz0
        arms[name] = {"time_to_tol_ms": round(statistics.median(sol), 3), "reps": reps,
                      "time_to_tol_ms_min": round(min(sol), 3), "time_to_tol_ms_max": round(max(sol), 3),
                      "setup_ms": round(setup_ms, 3), "iterations": info.iterations, "resets": info.resets,
                      "conv_factor": round(info.conv_factor, 4), "final_relres": info.final_relres,
                      "operator_complexity": round(oc, 4),
                      "vcycle_GBps": round(vby / (vms * 1e-3) / 1e9, 1) if vms > 0 else None,
                      "eager_breakdown_ms": {"total": round(eager_ms, 3), "vcycle_kernels": round(vms, 3),
                                             "pcg_kernels": round(pms, 3),
                                             "reintroduction_sparsify_and_prep": round(reint, 3),
                                             "other_host_and_checks": round(eager_ms - vms - pms - reint, 3)},
                      "nnz_per_level": [h.level_stats(l)["nnz_operator"] for l in range(h.num_levels)]}
        del h
    g0 = arms["galerkin"]["time_to_tol_ms"]
    for v in arms.values():
        v["speedup_vs_galerkin"] = round(g0 / v["time_to_tol_ms"], 3)
    return arms


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "poisson3d7":
        import torch

        from paper_1512_04629_gb300 import build

        build.build()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        {"poisson3d27": run_poisson3d27, "lognormal-batched": run_lognormal_batched, "serving": run_serving,
         "lump": run_lump, "aniso": run_aniso}[args.workload](args)
        return
    import numpy as np
    import torch

    import amg_inputs as gen
    import paper_1512_04629_gb300 as amg
    from paper_1512_04629_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    amg.lib()

    A = gen.poisson3d_7pt(args.grid)
    b = gen.rhs_uniform(A.n, 1)
    rp = torch.from_numpy(A.rowptr).cuda()
    ci = torch.from_numpy(A.col).cuda()
    va = torch.from_numpy(A.val).cuda()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    A_dev = amg.amg.csr_struct(rp, ci, va)
    gamma = [0.0, args.gamma]
    hopts = {"lump": amg.LUMP_STRONG if args.lump == "strong" else amg.LUMP_DIAG,
             "krylov": amg.KRYLOV_GMRES if args.krylov == "gmres" else amg.KRYLOV_CG}
    torch.cuda.synchronize()

    def step(timing=False):
        h = amg.Hierarchy.setup(A_dev, **hopts, gamma=gamma, use_graph=0 if args.eager else 1,
                                setup_timing=1 if timing else 0)
        if timing:
            setup_phases.append(collect_setup_timing(h, h.num_levels))
            h.timing_reset()
            h.timing_enable(True)
        x, info = h.solve(bd, xd, tol=args.tol)
        return h, info

    setup_phases = []

    if args.ncu_setup:
        h = amg.Hierarchy.setup(A_dev, **hopts, gamma=gamma, use_graph=0)
        del h
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.cudart().cudaProfilerStart()
        e0.record()
        h = amg.Hierarchy.setup(A_dev, **hopts, gamma=gamma, use_graph=0)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"ncu_setup": True, "levels": h.num_levels, "setup_ms": round(e0.elapsed_time(e1), 3)}))
        return

    if args.ncu_solve:
        h = amg.Hierarchy.setup(A_dev, **hopts, gamma=gamma, use_graph=0)
        h.solve(bd, xd, tol=args.tol)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        _, info = h.solve(bd, xd, tol=args.tol)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"ncu_solve": True, "iterations": info.iterations, "levels": h.num_levels}))
        return

    for _ in range(args.warmup):
        h, info = step()
        assert info.status == 0, info.as_dict()
        del h
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timings = {}
    its = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = amg.kernel_launches()
    ev0.record(stream)
    for _ in range(args.steps):
        h, info = step()
        its.append(info.iterations)
        assert info.status == 0 and info.final_relres <= args.tol, info.as_dict()
        del h
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = amg.kernel_launches() - launches0
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    # per-kernel CUDA-event pass over the same steps (eager launches with an
    # event pair around each solve-phase kernel on the launching stream)
    for _ in range(max(1, min(args.steps, 5))):
        h, info = step(timing=True)
        for r in collect_timing(h, h.num_levels):
            key = (r["kind"], r["level"])
            t = timings.setdefault(key, {"launches": 0, "ms": 0.0, "bytes": 0.0})
            t["launches"] += r["launches"]
            t["ms"] += r["ms"]
            t["bytes"] += r["bytes"]
        last_h = h
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    value = world * args.steps / elapsed
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # hierarchy shape of the timed configuration
    levels = []
    for l in range(last_h.num_levels):
        st = last_h.level_stats(l)
        levels.append({"n": st["n"], "nnz_galerkin": st["nnz_galerkin"], "nnz_operator": st["nnz_operator"],
                       "spmv": amg.SPMV_NAMES.get(st["spmv_variant"], "?"),
                       "spmv_P": amg.SPMV_NAMES.get(st["spmv_variant_p"], "-"),
                       "spmv_R": amg.SPMV_NAMES.get(st["spmv_variant_r"], "-"),
                       "bytes_per_cycle": st["bytes_per_cycle"]})

    # roofline of the dominant solve-phase kernel
    peak, peak_kind = measured_peak()
    dom_key = max(timings, key=lambda k: timings[k]["ms"])
    dom = timings[dom_key]
    per_launch_bytes = dom["bytes"] / dom["launches"]
    avg_ms = dom["ms"] / dom["launches"]
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    traffic = None
    tr = ncu_traffic().get(f"{dom_key[0]}_L{dom_key[1]}")
    if tr is not None:
        rows_cap, nnz_cap, bytes_cap = tr
        n_dom = levels[dom_key[1]]["n"]
        traffic = bytes_cap * (n_dom / rows_cap) if rows_cap else None
    roofline = {"kernel": f"{dom_key[0]} level {dom_key[1]}", "bound": "hbm", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
                "launches": dom["launches"]}
    # the second ceiling of these kernels: the FP64 pipe (GB300 has 2 FP64 FMA per clock per SM)
    lv = levels[dom_key[1]]
    ops = fp64_ops_per_launch(dom_key[0], dom_key[1], lv["n"], lv["nnz_operator"] if dom_key[1] > 0 else lv["nnz_galerkin"],
                              "fp64")
    if ops is not None:
        clk = (clocks or {}).get("sm_mhz") or 2070.0
        fpeak = FP64_FMA_PER_CLK_SM * GB300_SMS * clk * 1e6 / 1e12
        fach = ops / (avg_ms * 1e-3) / 1e12
        roofline["fp64"] = {"ops_per_launch": ops, "achieved": fach, "peak": fpeak, "unit": "Tops/s",
                            "frac": fach / fpeak,
                            "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x sampled SM clock"}
    vcycle_ms = sum(v["ms"] for k, v in timings.items() if k[0] not in ("pcg_Ap_dot", "pcg_vector"))
    vcycle_bytes = sum(v["bytes"] for k, v in timings.items() if k[0] not in ("pcg_Ap_dot", "pcg_vector"))
    per_level_ms = {}
    for (kind, lv), v in timings.items():
        per_level_ms[lv] = per_level_ms.get(lv, 0.0) + v["ms"]
    steps_timed = max(1, min(args.steps, 5))
    per_level_ms = {f"L{lv}": round(ms / steps_timed, 3) for lv, ms in sorted(per_level_ms.items())}
    kernels = sorted(({"kernel": f"{k[0]} L{k[1]}", "launches": v["launches"], "ms": round(v["ms"], 4),
                       "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None}
                      for k, v in timings.items()), key=lambda r: -r["ms"])[:12]

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(a).pin_memory() for a in (A.rowptr, A.col, A.val, b)]
        xh = torch.zeros(A.n, dtype=torch.float64).pin_memory()
        A_host = amg.amg.csr_struct(hp[0].numpy(), hp[1].numpy(), hp[2].numpy())
        bh = hp[3].numpy()
        xn = xh.numpy()
        ke = max(1, min(args.steps, 5))
        h = amg.Hierarchy.setup(A_host, **hopts, gamma=gamma)
        h.solve(bh, xn, tol=args.tol)
        del h
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            h = amg.Hierarchy.setup(A_host, **hopts, gamma=gamma)
            _, info = h.solve(bh, xn, tol=args.tol)
            assert info.status == 0
            del h
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = A.rowptr.nbytes + A.col.nbytes + A.val.nbytes + b.nbytes
        e2e = {"value": ke / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(xn.nbytes),
               "steps": ke}

    # arms (outside the timed region): solve-only time to 1e-8 per hierarchy
    arms = None
    if not args.no_arms:
        arms = solve_arms(args, A_dev, A.nnz, bd, xd, stream)

    comm = None
    if not args.no_arms:
        comm = communication(A_dev)
    setup_roof = None
    if setup_phases:
        setup_roof = setup_roofline(last_h, _median_phases(setup_phases))

    # the other configurations of the metric, each with its own config and clocks
    legs = None
    if world == 1 and not args.no_legs:
        legs = {}
        for name, fn in (("c3_precision_27pt_192", lambda: leg_c3(args)),
                         ("c4_batched_lognormal_160", lambda: leg_c4(args)),
                         ("c5_serving", lambda: leg_c5(args, seconds=args.leg_serve_seconds))):
            t0 = time.perf_counter()
            try:
                legs[name] = fn()
            except Exception as e:  # reported, not hidden: the headline above stands on its own
                legs[name] = {"error": f"{type(e).__name__}: {e}"}
            legs[name]["wall_s"] = round(time.perf_counter() - t0, 1)
            torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline_leg(args, A, b)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args),
        "iterations": statistics.median(its), "levels": levels,
        "roofline": roofline, "vcycle_GBps": vcycle_bytes / (vcycle_ms * 1e-3) / 1e9 if vcycle_ms else None,
        "top_kernels": kernels, "solve_ms_per_level": per_level_ms, "setup_phases_ms": _median_phases(setup_phases),
        "setup_roofline": setup_roof,
        "e2e": e2e, "cpu_baseline": cpu, "arms": arms, "communication": comm, "legs": legs, "clocks": clocks,
        "gpu_launches": launches,
    }
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
