#!/usr/bin/env python
"""Benchmark of the time-parallel inexact Uzawa solver on one GB300 per rank.

Workload (the metric's configuration): 2-D heat equation on the unit square, 5-point finite
differences on a 255 x 255 interior grid, N_t = 1024 implicit-Euler steps, T = 1,
a = 1 + 0.5 sin(2 pi x) sin(2 pi y) cos(2 pi t), f i.i.d. U(-1,1) per space-time node
(SplitMix64, seed 1), u0 = 0; plain FP64 method (66,585,600 space-time DOFs).

A step is one complete solve from u = p = 0 to ||F - B u|| / ||F|| <= 1e-8 (every kernel of the
hot path: residuals, V-cycles, DSTs, block solves, updates, reductions).  `value` is space-time
DOFs per second with the data resident in HBM; `e2e` repeats the measurement through the C ABI
with the source in pinned host memory and the solution copied back every step.  Each space-time
vector (533 MB) is larger than the 129 MB L2, so no flush is needed between steps.

Multi-GPU: every rank solves its own copy of the workload (the solves share nothing);
`value` is the DOFs of all ranks over the slowest rank's time (weak scaling).

`--impl reference` times the CPU oracle (sequential implicit Euler with banded Cholesky per
step) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "space-time DOFs/s to 1e-8 rel residual"
WORKLOAD = "heat2d_fd5_255x255_Nt1024_T1_fp64_plain"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--omega", type=float, default=0.5)
    ap.add_argument("--max-it", type=int, default=2000)
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--nt", type=int, default=1024)
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="override the workload's precision (profiling runs)")
    ap.add_argument("--workload", default="heat2d", choices=["heat2d", "heat1d", "heat3d", "batch", "serve"])
    ap.add_argument("--problems", type=int, default=512, help="batch: number of problems")
    ap.add_argument("--batch-mode", default="waves", choices=["waves", "server"],
                    help="batch: pt_solve_batch over memory waves, or all problems submitted at once "
                         "to the continuous-batching server (finished solves replaced at once)")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per arrival rate")
    ap.add_argument("--rates", default="0.5,0.9,1.1", help="serve: arrival rates as fractions of capacity")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
        return rank, ws, local, dist
    return rank, ws, local, None


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over the ranks (x itself without a process group): the timed region
    of a multi-GPU run is the slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp64_peak_tflops(peaks):
    """FP64 pipe peak of the GB300: 152 SMs x 2 FP64 FMA lanes per clock x 2 flop x max SM clock."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


def fp64_flops_per_launch(name, dim, n, N):
    """Algorithmic FP64 flops of one launch of a kernel of the FP64 path (2-D workloads).

    Transforms use the standard count for a real-input FFT of length L, 2.5 L log2 L per line; a
    DST-I of n points is one such FFT of length M = n + 1, the temporal DST one of length N.
    Stencil kernels count the flops of the formulas they evaluate per interior point (face
    coefficients a0 + c g g: 2 each; 5-point variable-coefficient stencil: 11)."""
    if dim != 2:
        return None
    M = n + 1
    pts = float(N) * n * n
    fft_M = 2.5 * M * math.log2(M)
    if name == "dsti_cols_scale":   # two y-transforms of every x-column + the product with the
        return N * n * 2 * fft_M + 1.0 * pts  # precomputed block-solve factor
    if name == "dsti_rows":
        return N * n * fft_M
    if name in ("dst_forward", "dst_inverse"):  # N-point transform of every spatial point + twiddles
        return n * n * (2.5 * N * math.log2(N) + 6.0 * N)
    if name == "hsolve_y":          # per (k, x-frequency) column: two Thomas eliminations (6 flops
        return 16.0 * pts            # each: multiply-add, multiply) and the tridiagonal product (4)
    if name == "resid_bres":        # bres (faces 8, stencil 11, K and F 3, norm 2) + r_p (13)
        return 37.0 * pts
    if name == "mg2_up":            # 3 launches (levels 0, 1, 2): prolong 5, stencil 19, smoothing 4
        return 28.0 * pts * (1 + 0.25 + 0.0625) / 3
    if name == "mg2_down":          # x1 1, stencil 19, residual 1, restriction 9/4
        return 23.25 * pts * (1 + 0.25 + 0.0625) / 3
    return None


# Fused-minimum algorithmic bytes per DOF per Uzawa iteration (outer passes at 8 B, preconditioner
# passes at 8 B or 4 B, three V(1,1) cycles): the model the path-level HBM roofline is quoted on.
HBM_MODEL_BYTES = {("fp64", 2): 368.0, ("mixed", 2): 232.0, ("fp64", 3): 336.0, ("mixed", 3): 216.0}


def path_roofline(prof, dims, iterations, value, precision, peaks, steps):
    """Whole-solve bounds in DOFs/s: HBM bandwidth over the byte model, and (FP64 path) the FP64
    pipe over the algorithmic flops of the modelled kernels; `frac` = value / the smaller."""
    try:
        dim, n, N = dims
        dofs = float(N) * n ** dim
        out = {}
        b = HBM_MODEL_BYTES.get((precision, dim))
        if b:
            out["hbm_model_bytes_per_dof_iteration"] = b
            out["hbm_bound_dofs_per_s"] = peaks["hbm_gbs"] * 1e9 / (b * iterations)
        if precision == "fp64":
            fl = 0.0
            for k, v in prof.items():
                f = fp64_flops_per_launch(k, dim, n, N)
                if f is not None:
                    fl += f * v["launches"] / steps
            if fl > 0:
                out["fp64_flops_per_dof_iteration"] = fl / dofs / iterations
                out["fp64_bound_dofs_per_s"] = fp64_peak_tflops(peaks) * 1e12 * dofs / fl
        bounds = [v for k, v in out.items() if k.endswith("_bound_dofs_per_s")]
        if not bounds:
            return None
        out["bound"] = "hbm" if min(bounds) == out.get("hbm_bound_dofs_per_s") else "fp64"
        out["frac"] = value / min(bounds)
        return out
    except Exception:
        return None


def roofline_of(prof, name, bound_fp64, dims, peaks, peak_src, tr):
    d = prof[name]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
    share = d["ms"] / sum(v["ms"] for v in prof.values())
    base = {"kernel": name, "traffic": tr.get((name, WORKLOAD)),
            "algorithmic_bytes_per_launch": d["bytes"] / max(d["launches"], 1),
            "avg_launch_ms": per_launch_ms, "share": share}
    fl = fp64_flops_per_launch(name, *dims) if bound_fp64 else None
    if fl is not None:
        tf = fl / (per_launch_ms / 1e3) / 1e12
        pk = fp64_peak_tflops(peaks)
        base.update({"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk,
                     "algorithmic_flops_per_launch": fl, "hbm_GBps": gbs,
                     "peak_source": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x %.0f MHz (%s clock)"
                                    % (float(peaks.get("sm_max_mhz", 2070.0)), peak_src)})
    else:
        base.update({"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_src})
    return base


def traffic_table():
    """DRAM bytes per launch from the committed ncu summary, valid only for the kernel source
    it was measured on (checked by hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    csrc = os.path.join(ROOT, "paper_1802_08126_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, fn), "rb") as fh:
                h.update(fh.read())
    current = h.hexdigest()[:16]
    table = {}
    try:
        with open(path) as fh:
            for ln in fh:
                ln = ln.strip()
                if not ln or ln.startswith("#"):
                    continue
                parts = ln.split()
                if len(parts) >= 4 and parts[3] == current:
                    table[(parts[0], parts[1])] = float(parts[2])
    except FileNotFoundError:
        pass
    return table


def cpu_sample(prob, seconds, f=None):
    """Oracle implicit Euler on the first k steps of the workload; returns (dofs/s, k, secs, cores)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    if f is None:
        f = S.source(prob, steps=min(prob.N, 64))
    method = "cg" if prob.dim == 3 else "cholesky"  # the 3-D band is too wide to factor
    u0 = S.initial(prob)
    t0 = time.perf_counter()
    oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=1, method=method)
    one = time.perf_counter() - t0
    k = int(max(1, min(f.shape[0], seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=k, method=method)
    secs = time.perf_counter() - t0
    return k * prob.ns / secs, k, secs, cores, method


def cpu_single_thread(prob, f, method, cores):
    """The oracle on one host thread: DOFs/s of its first step (then all cores again)."""
    import oracle
    try:
        u0 = S.initial(prob)
        t0 = time.perf_counter()
        oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=1, method=method,
                              threads=1)
        secs = time.perf_counter() - t0
        return {"value": prob.ns / secs, "unit": "DOF/s", "cores": 1, "sample": "first step (%.2f s)" % secs}
    except Exception:
        return None
    finally:
        oracle.implicit_euler(prob.dim, [1] * prob.dim, 1, prob.T, prob.coeff, np.zeros(1), None, threads=cores)


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return 0
    prob = S.heat2d_uniform(args.n, args.nt)
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    f = S.source(prob, steps=4)
    per_step = 2  # implicit-Euler steps of the workload per timed reference step
    for _ in range(args.warmup):
        oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, steps=per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, steps=per_step)
    secs = time.perf_counter() - t0
    value = args.steps * per_step * prob.ns / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [prob.n[0]] * 2, "N_t": prob.N,
                                        "tol": args.tol},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "DOF/s", "cores": cores,
                         "sample": "%d implicit-Euler steps (banded Cholesky, 255^2) per timed step"
                                   % per_step},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_batch_problem(ptu, p, precision="mixed"):
    P = ptu.Problem(p.dim, p.n, p.N, p.T, p.coeff, None, None, precision=precision)
    P.set_rhs_uniform(p.seed)
    return P


def run_batch(args, rank, ws, dist):
    """512 independent 2-D problems (grids 31..255, N_t log-uniform in [16, 2048], c ~ U(0, 0.8),
    k in {1..4}, f ~ U(-1,1) from per-problem seeds), mixed precision, solved with pt_solve_batch in
    waves that fit the device memory; DOFs/s over the solve time of all waves."""
    import torch

    import paper_1802_08126_gb300 as ptu
    from paper_1802_08126_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local_rank())
    probs = [S.batch_problem(i + rank * args.problems) for i in range(args.problems)]
    # warm-up: three small batches of the smallest problems
    small = sorted(probs, key=lambda p: p.dofs)[:8]
    for _ in range(max(args.warmup, 3)):
        Ps = [make_batch_problem(ptu, p) for p in small]
        ptu.solve_batch(Ps, args.tol, args.max_it)
        for P in Ps:
            P.close()
    total_dofs = sum(p.dofs for p in probs)
    clocks = ClockSampler(local_rank())
    clocks.start()
    launches0 = ptu.launch_count()
    solve_s, waves, its, statuses, i = 0.0, 0, [], [], 0
    if args.batch_mode == "server":
        # every problem submitted at t = 0; the server admits by memory and refills as solves end
        with ptu.Server() as sv:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tickets = [sv.submit(p.dim, p.n, p.N, p.T, p.coeff, None, seed=p.seed, tol=args.tol,
                                 max_it=args.max_it, precision="mixed") for p in probs]
            for t in tickets:
                stt, it = sv.wait(t)
                its.append(it)
                statuses.append(stt)
            solve_s = time.perf_counter() - t0
        waves = 0
        i = len(probs)
    while i < len(probs):
        free, _ = torch.cuda.mem_get_info()
        budget = free - (24 << 30)
        Ps, used = [], 0
        while i < len(probs):
            est = ptu.estimate_bytes(probs[i].dim, probs[i].n, probs[i].N, "mixed")
            if Ps and used + est > budget:
                break
            Ps.append(make_batch_problem(ptu, probs[i]))
            used += est
            i += 1
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, sts = ptu.solve_batch(Ps, args.tol, args.max_it)
        torch.cuda.synchronize()
        solve_s += time.perf_counter() - t0
        its += it
        statuses += sts
        waves += 1
        for P in Ps:
            P.close()
    launches = ptu.launch_count() - launches0
    clk = clocks.stop()
    solve_s = max_over_ranks(solve_s, dist)
    if rank == 0:
        line = {
            "metric": METRIC + " (batched)", "value": ws * total_dofs / solve_s, "unit": "DOF/s",
            "n_gpus": ws, "steps": 1, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * solve_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": "batch%d_heat2d_mixed" % args.problems, "problems": len(probs),
                       "dofs_per_gpu": total_dofs, "tol": args.tol, "waves": waves, "mode": args.batch_mode,
                       "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
                       "converged": int(sum(1 for x in statuses if x == 0)), "precision": "mixed",
                       "l2": "inputs larger than L2 for most problems"},
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, ws, dist):
    """Poisson arrivals of requests drawn from the batch distribution, served by pt_server at
    several arrival rates given as fractions of the measured capacity; p50/p99 latency."""
    import torch

    import paper_1802_08126_gb300 as ptu
    from paper_1802_08126_gb300 import build
    if rank != 0:
        return 0
    build.build()
    torch.cuda.set_device(local_rank())
    rng = np.random.default_rng(5)
    pool = [S.batch_problem(i, master_seed=5) for i in range(4 * args.requests)]
    mean_dofs = float(np.mean([p.dofs for p in pool]))
    # capacity: DOFs/s of one batch of the first requests
    cap_probs = pool[:32]
    Ps = [make_batch_problem(ptu, p) for p in cap_probs]
    ptu.solve_batch(Ps, args.tol, args.max_it)
    for P in Ps:
        P.set_rhs_uniform(cap_probs[Ps.index(P)].seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ptu.solve_batch(Ps, args.tol, args.max_it)
    torch.cuda.synchronize()
    capacity = sum(p.dofs for p in cap_probs) / (time.perf_counter() - t0)
    for P in Ps:
        P.close()
    results = []
    for frac in [float(x) for x in args.rates.split(",")]:
        lam = frac * capacity / mean_dofs  # requests per second
        reqs = [pool[int(k)] for k in rng.integers(0, len(pool), args.requests)]
        gaps = rng.exponential(1.0 / lam, args.requests)
        with ptu.Server() as sv:
            tickets = []
            t_start = time.perf_counter()
            t_next = t_start
            for p, g in zip(reqs, gaps):
                t_next += g
                delay = t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(sv.submit(p.dim, p.n, p.N, p.T, p.coeff, None, seed=p.seed, tol=args.tol,
                                         max_it=args.max_it, precision="mixed"))
            ok = 0
            for t in tickets:
                st, it = sv.wait(t)
                ok += st == 0
            st_ = sv.stats()
            wall = time.perf_counter() - t_start
        results.append({"rate_frac": frac, "req_per_s": lam, "p50_ms": st_["p50_ms"], "p99_ms": st_["p99_ms"],
                        "dofs_per_s": st_["dofs_per_s"], "completed": st_["completed"], "converged": ok,
                        "wall_s": wall})
    best = max(r["dofs_per_s"] for r in results)
    line = {
        "metric": "p50/p99 solve latency and DOFs/s under Poisson arrivals", "value": best, "unit": "DOF/s",
        "n_gpus": 1, "steps": len(results), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "serve_heat2d_mixed", "requests_per_rate": args.requests, "tol": args.tol,
                   "capacity_dofs_per_s": capacity, "mean_request_dofs": mean_dofs},
        "rates": results,
    }
    print(json.dumps(line), flush=True)
    return 0


def local_rank():
    return int(os.environ.get("LOCAL_RANK", "0"))


def main():
    args = parse()
    rank, ws, local, dist = dist_init(args)
    if args.impl == "reference":
        return run_reference(args, rank, ws, dist)
    if args.workload == "batch":
        return run_batch(args, rank, ws, dist)
    if args.workload == "serve":
        return run_serve(args, rank, ws, dist)

    import torch

    import paper_1802_08126_gb300 as ptu
    from paper_1802_08126_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if args.workload == "heat1d":
        prob = S.heat1d_mms(63, 64)
        solver, base_prec = "exact", "fp64"
    elif args.workload == "heat3d":
        prob = S.heat3d_bumps(127, 256)
        solver, base_prec = "mg", "mixed"  # the 3-D workload is specified in mixed precision
    else:
        prob = S.heat2d_uniform(args.n, args.nt)
        solver, base_prec = "mg", "fp64"
    if args.precision:
        base_prec = args.precision
    global WORKLOAD
    WORKLOAD = {"heat1d": "heat1d_fd3_63_Nt64_T1_fp64_exact", "heat3d": "heat3d_fd7_127^3_Nt256_T2",
                "heat2d": WORKLOAD}[args.workload]
    dofs = prob.dofs
    f = S.source(prob)
    u0 = S.initial(prob)
    P = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision=base_prec,
                    omega=args.omega, solver=solver)
    variant = "fp64" if base_prec == "mixed" else "mixed"

    def solve_once(Pr):
        st, it, hist = Pr.solve(args.tol, args.max_it)
        if st != 0:
            raise RuntimeError("solve did not converge: status %d after %d iterations" % (st, it))
        return it, hist[-1]

    for _ in range(args.warmup):
        iters, res = solve_once(P)

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ptu.launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    its = []
    for _ in range(args.steps):
        it, res = solve_once(P)
        its.append(it)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ptu.launch_count() - launches0
    clk = clocks.stop()
    # the same steps again with a CUDA event pair around every kernel (graphs off): per-kernel
    # times for the breakdown and the roofline (the value above is measured without them)
    ptu.profile_reset()
    ptu.profile_enable(True)
    torch.cuda.synchronize()
    e0p, e1p = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0p.record()
    for _ in range(args.steps):
        solve_once(P)
    e1p.record()
    torch.cuda.synchronize()
    ms_prof = e0p.elapsed_time(e1p)
    ptu.profile_enable(False)
    prof = ptu.profile_totals()
    ms = max_over_ranks(ms, dist)
    value = ws * dofs * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (largest share of the timed region): FP64-pipe bound for the
    # FP64 kernels of the FP64 path, HBM bound otherwise
    peaks, peak_src = load_peaks()
    tr = traffic_table()
    dims = (prob.dim, prob.n[0], prob.N)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])[0] if prof else None
    roof = roofline_of(prof, dom, base_prec == "fp64", dims, peaks, peak_src, tr) if dom else None
    phases = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                  "GBps": v["bytes"] / max(v["ms"], 1e-9) / 1e6}
              for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    # end to end through the C ABI: pinned host source in, solution out, every step
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(f).pin_memory().numpy()
        uh = torch.empty((prob.N, prob.ns), dtype=torch.float64).pin_memory().numpy()
        P.set_rhs(fh, u0)
        P.solve(args.tol, args.max_it, u_out=uh)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.set_rhs(fh, u0)
            st, it, hist = P.solve(args.tol, args.max_it, u_out=uh)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        barrier()
        secs = max_over_ranks(secs, dist)
        e2e = {"value": ws * dofs * args.steps / secs, "unit": "DOF/s",
               "h2d_bytes_per_step": int(fh.nbytes), "d2h_bytes_per_step": int(uh.nbytes + 8 * (it + 1))}
        u64 = uh.copy()
    else:
        u64 = np.zeros((prob.N, prob.ns))
        P.solve(args.tol, args.max_it, u_out=u64)

    # the other precision on the same workload (mixed for the FP64 workloads, FP64 for the 3-D one)
    mixed = None
    if not args.no_mixed:
        Pm = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision=variant,
                         omega=args.omega, solver=solver)
        vsteps = args.steps if variant == "mixed" else 1
        if variant == "mixed":
            solve_once(Pm)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mits = []
        for _ in range(vsteps):
            it, res = solve_once(Pm)
            mits.append(it)
        e1.record()
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1)
        # per-kernel breakdown from one more solve with kernel events
        ptu.profile_reset()
        ptu.profile_enable(True)
        solve_once(Pm)
        torch.cuda.synchronize()
        ptu.profile_enable(False)
        vprof = ptu.profile_totals()
        um = np.zeros((prob.N, prob.ns))
        Pm.solve(args.tol, args.max_it, u_out=um)
        Pm.close()
        mms = max_over_ranks(mms, dist)
        vdom = max(vprof.items(), key=lambda kv: kv[1]["ms"])[0] if vprof else None
        mixed = {"precision": variant, "value": ws * dofs * vsteps / (mms / 1e3), "unit": "DOF/s",
                 "roofline": roofline_of(vprof, vdom, variant == "fp64", dims, peaks, peak_src, tr)
                 if vdom else None,
                 "ms_per_step": mms / vsteps, "iterations": mits[-1],
                 "rel_l2_mixed_vs_fp64_path": float(np.linalg.norm(um - u64) / np.linalg.norm(u64)),
                 "kernels": {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"],
                                 "GBps": v["bytes"] / max(v["ms"], 1e-9) / 1e6}
                             for k, v in sorted(vprof.items(), key=lambda kv: -kv[1]["ms"])}}
    P.close()

    # the Krylov-accelerated form (flexible GMRES(10) preconditioned by one Uzawa step), FP64 2-D
    krylov = None
    if not args.no_mixed and base_prec == "fp64" and prob.dim == 2:
        Pk = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="fp64",
                         omega=args.omega, solver=solver, krylov=10)
        solve_once(Pk)
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        kits = []
        for _ in range(args.steps):
            it, res = solve_once(Pk)
            kits.append(it)
        k1.record()
        torch.cuda.synchronize()
        kms = max_over_ranks(k0.elapsed_time(k1), dist)
        uk = np.zeros((prob.N, prob.ns))
        Pk.solve(args.tol, args.max_it, u_out=uk)
        Pk.close()
        krylov = {"solver": "FGMRES(10), right preconditioner: one inexact Uzawa step",
                  "value": ws * dofs * args.steps / (kms / 1e3), "unit": "DOF/s", "ms_per_step": kms / args.steps,
                  "iterations": kits[-1],
                  "rel_l2_vs_uzawa_solution": float(np.linalg.norm(uk - u64) / np.linalg.norm(u64))}

    # the same workload on quasi-uniform random time steps (ratio <= 1.5, §2 eq. 2.1-2.2), FP64
    nonuniform = None
    if not args.no_mixed and base_prec == "fp64" and prob.dim == 2:
        taus = S.random_steps(prob.N, prob.T, 1, 0.5)
        Pn = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="fp64", solver=solver,
                         taus=taus)
        solve_once(Pn)
        torch.cuda.synchronize()
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record()
        nits = []
        for _ in range(args.steps):
            it, res = solve_once(Pn)
            nits.append(it)
        n1.record()
        torch.cuda.synchronize()
        nms = max_over_ranks(n0.elapsed_time(n1), dist)
        Pn.close()
        nonuniform = {"steps": "tau_n = T w_n / sum w, w_n = 1 + 0.5 U_n (SplitMix64 seed 1), max/min %.3f"
                               % (taus.max() / taus.min()),
                      "omega": "default: 1.5 / (1 + alpha), alpha of eq. 2.2 with the step ratios",
                      "h_solver": "exact, by spatial sine transforms (reference: the time-mean coefficient)",
                      "value": ws * dofs * args.steps / (nms / 1e3), "unit": "DOF/s",
                      "ms_per_step": nms / args.steps, "iterations": nits[-1]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, k, secs, cores, method = cpu_sample(prob, args.cpu_seconds, f[:64])
        cpu = {"value": v, "unit": "DOF/s", "cores": cores, "kind": "oracle",
               "sample": "first %d of %d implicit-Euler steps, %s per step (%.1f s)"
                         % (k, prob.N, "banded Cholesky" if method == "cholesky" else "CG to 1e-14", secs),
               "single_thread": cpu_single_thread(prob, f[:64], method, cores)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if base_prec == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(prob.n), "precision": base_prec, "N_t": prob.N, "T": prob.T,
                       "dofs_per_gpu": dofs, "tol": args.tol, "omega": args.omega,
                       "iterations": its[-1],
                       "spatial_solver": "exact tridiagonal" if solver == "exact"
                       else "V(1,1) geometric multigrid (1 cycle per A_n solve, 2 per H_k solve)",
                       "l2": "inputs larger than L2 (533 MB per space-time vector)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "path_roofline": path_roofline(prof, dims, its[-1], value, base_prec, peaks, args.steps),
            "ms_per_step_with_kernel_events": ms_prof / args.steps,
            "clocks": clk, ("fp64_path" if variant == "fp64" else "mixed"): mixed, "krylov": krylov,
            "nonuniform_steps": nonuniform,
            "kernels": phases,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
