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
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests per arrival rate")
    ap.add_argument("--rates", default="0.25,0.5,0.75,0.9,1.1", help="serve: arrival rates as fractions of capacity")
    ap.add_argument("--autotune", action="store_true",
                    help="batch / serve: tune the launch configurations (pt_options.autotune = 1)")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--no-3d", action="store_true", help="leave out the 3-D entry")
    ap.add_argument("--batch-sample", type=int, default=64,
                    help="problems of the batch distribution in the default line's batch entry (0: none)")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="run exactly this many iterations of one solve of the workload and exit (for ncu)")
    ap.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
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


def r4(x):
    """x rounded to 4 significant digits (keeps the JSON line short)."""
    if isinstance(x, bool) or not isinstance(x, float) or x == 0.0 or not math.isfinite(x):
        return x
    return float("%.4g" % x)


def compact(d):
    """A copy of dict d with its float values rounded by r4 (nested dicts too)."""
    if not isinstance(d, dict):
        return d
    return {k: (compact(v) if isinstance(v, dict) else r4(v)) for k, v in d.items()}


# ---- the CPU leg: the oracle on a bounded sample, in a fresh process --------------------------

def workload_problem(name):
    """The synthetic problem of a named workload (shared by the GPU arm and the CPU leg)."""
    if name == "heat1d":
        return S.heat1d_mms(63, 64)
    if name == "heat3d":
        return S.heat3d_bumps(127, 256)
    if name.startswith("batch"):
        return S.batch_problem(int(name[5:]))
    if name.startswith("heat2d"):
        n, N = (int(v) for v in name[6:].split("x")) if "x" in name else (255, 1024)
        return S.heat2d_uniform(n, N)
    raise ValueError(name)


def cpu_leg_main(spec):
    """Child-process body of the CPU leg: the oracle (sequential implicit Euler) on the first k steps
    of the workload, k chosen for about `seconds` of work (at most `max_steps`); the steps are
    written to `out` for the parity check and the timing is printed as one JSON line.  The child
    imports neither torch nor the CUDA library, as the reference arm does not."""
    import oracle
    oracle.build()
    prob = workload_problem(spec["workload"])
    cores = oracle.max_threads()
    kmax = int(min(prob.N, spec.get("max_steps", prob.N)))
    f = S.source(prob, steps=kmax)
    u0 = S.initial(prob)
    method = "cg" if prob.dim == 3 else "cholesky"  # the 3-D band is too wide to factor
    t0 = time.perf_counter()
    oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=1, method=method)
    one = time.perf_counter() - t0
    k = int(max(1, min(kmax, spec["seconds"] / max(one, 1e-4))))
    t0 = time.perf_counter()
    u = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=k, method=method)
    secs = time.perf_counter() - t0
    np.save(spec["out"], u)
    res = {"value": k * prob.ns / secs, "k": k, "secs": secs, "cores": cores, "method": method}
    if spec.get("single_thread"):
        t0 = time.perf_counter()
        oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, steps=1, method=method,
                              threads=1)
        st = time.perf_counter() - t0
        res["single_thread"] = {"value": prob.ns / st, "cores": 1, "sample": "first step (%.2f s)" % st}
    print(json.dumps(res), flush=True)
    return 0


def cpu_leg(workload, seconds, max_steps, single_thread=False):
    """Run the CPU leg in a fresh interpreter; returns (timing dict, oracle steps [k][ns]), or
    (None, None) when it fails (the CPU leg is a reported baseline, not the measurement)."""
    import tempfile
    fd, out = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    spec = {"workload": workload, "seconds": seconds, "max_steps": max_steps, "out": out,
            "single_thread": single_thread}
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", json.dumps(spec)],
                           capture_output=True, text=True, timeout=900, cwd=ROOT)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            sys.stderr.write("cpu leg %s failed:\n%s\n" % (workload, r.stderr[-2000:]))
            return None, None
        return json.loads(lines[-1]), np.load(out)
    except Exception as exc:
        sys.stderr.write("cpu leg %s failed: %s\n" % (workload, exc))
        return None, None
    finally:
        try:
            os.remove(out)
        except OSError:
            pass


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cpu_baseline_entry(res, prob):
    if res is None:
        return None
    out = {"value": res["value"], "unit": "DOF/s", "cores": res["cores"], "kind": "oracle",
           "sample": "first %d of %d implicit-Euler steps, %s per step (%.1f s), in a fresh process"
                     % (res["k"], prob.N, "banded Cholesky" if res["method"] == "cholesky" else "CG to 1e-14",
                        res["secs"])}
    if "single_thread" in res:
        out["single_thread"] = dict(res["single_thread"], unit="DOF/s")
    return out


def spatial_solver_label(dim, solver, h_solver):
    if solver == "exact":
        return "exact tridiagonal solves (A~_n and H_k)"
    a = "A~_n: one V(1,1) geometric-multigrid cycle per step; "
    if h_solver == "vcycle":
        return a + "H_k: two V(1,1) cycles per frequency"
    if dim == 2:
        return a + ("H_k: exact, spatial DST-I in x and tridiagonal eliminations in y (FP64), "
                    "DST-I in x and y (FP32)")
    return a + "H_k: exact, spatial DST-I along every axis"


def headline_config(prob, tol, omega, ws, precision="fp64", solver="mg"):
    return {"workload": WORKLOAD, "grid": list(prob.n), "precision": precision, "N_t": prob.N, "T": prob.T,
            "dofs_per_gpu": prob.dofs, "tol": tol, "omega": omega,
            "spatial_solver": spatial_solver_label(prob.dim, solver, "auto"),
            "l2": "inputs larger than L2 (%d MB per space-time vector)" % (prob.dofs * 8 >> 20),
            "parallelism": "replicas" if ws > 1 else "single"}


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
        "data": "synthetic", "config": headline_config(prob, args.tol, args.omega, ws),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "DOF/s", "cores": cores,
                         "sample": "%d implicit-Euler steps (banded Cholesky, 255^2) per timed step"
                                   % per_step},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0



def make_batch_problem(ptu, p, precision="mixed", autotune=0):
    P = ptu.Problem(p.dim, p.n, p.N, p.T, p.coeff, None, None, precision=precision, autotune=autotune)
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
                                 max_it=args.max_it, precision="mixed", autotune=1 if args.autotune else 0)
                       for p in probs]
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
            Ps.append(make_batch_problem(ptu, probs[i], autotune=1 if args.autotune else 0))
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
                       "autotune": bool(args.autotune), "loop": "device (conditional graph node)",
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
                                         max_it=args.max_it, precision="mixed",
                                         autotune=1 if args.autotune else 0))
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
                   "autotune": bool(args.autotune),
                   "capacity_dofs_per_s": capacity, "mean_request_dofs": mean_dofs},
        "rates": results,
    }
    print(json.dumps(line), flush=True)
    return 0


def local_rank():
    return int(os.environ.get("LOCAL_RANK", "0"))


def solve_timed(P, count, tol, max_it):
    """`count` solves from zero, CUDA events on the current stream; (ms per solve, iterations)."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    its = []
    for _ in range(count):
        st, it, hist = P.solve(tol, max_it)
        if st != 0:
            raise RuntimeError("solve did not converge: status %d after %d iterations" % (st, it))
        its.append(it)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / count, its[-1]


def kernel_profile(ptu, P, count, tol, max_it):
    """Per-kernel totals of `count` solves with an event pair around every kernel (graphs off)."""
    import torch
    ptu.profile_reset()
    ptu.profile_enable(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(count):
        P.solve(tol, max_it)
    e1.record()
    torch.cuda.synchronize()
    ptu.profile_enable(False)
    return ptu.profile_totals(), e0.elapsed_time(e1) / count


def dominant_roofline(prof, fp64, dims, peaks, peak_src, tr, short=False):
    if not prof:
        return None
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])[0]
    roof = roofline_of(prof, dom, fp64, dims, peaks, peak_src, tr)
    if short:
        roof = {k: roof[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "share")}
    return compact(roof)


def secondary(value, ms, it, rel, ksteps, roof, **extra):
    out = {"value": value, "unit": "DOF/s", "ms_per_solve": ms, "iterations": it,
           "rel_l2_vs_oracle": rel, "oracle_steps": ksteps}
    out.update(extra)
    if roof is not None:
        out["roofline"] = roof
    return compact(out)


def main():
    args = parse()
    if args.cpu_leg:
        return cpu_leg_main(json.loads(args.cpu_leg))
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

    def barrier():
        if dist is not None:
            dist.barrier()

    # the metric's workload (2-D, FP64); --workload / --precision / --n / --nt select another one for
    # profiling runs, which then report that workload alone
    global WORKLOAD
    wl = args.workload
    prec = args.precision or ("mixed" if wl == "heat3d" else "fp64")
    solver = "exact" if wl == "heat1d" else "mg"
    prob = workload_problem("heat2d%dx%d" % (args.n, args.nt) if wl == "heat2d" else wl)
    if (wl, prec, args.n, args.nt) != ("heat2d", "fp64", 255, 1024):
        WORKLOAD = "%s_%s_%s" % (wl, "x".join(str(v) for v in prob.n) + "_Nt%d" % prob.N, prec)
        args.no_extras, args.no_mixed = True, True
    dims = (prob.dim, prob.n[0], prob.N)
    dofs = prob.dofs
    f = S.source(prob)
    u0 = S.initial(prob)
    P = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision=prec, omega=args.omega,
                    solver=solver)
    if args.profile_iters > 0:
        # a fixed number of iterations (launch lists and counter captures), no measurement
        P.solve(0.0, args.profile_iters)
        torch.cuda.synchronize()
        P.close()
        return 0
    for _ in range(args.warmup):
        st, it, _ = P.solve(args.tol, args.max_it)
        if st != 0:
            raise RuntimeError("solve did not converge: status %d" % st)

    # ---- the timed region: K complete solves with F resident in HBM ----
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ptu.launch_count()
    barrier()
    ms, iters = solve_timed(P, args.steps, args.tol, args.max_it)
    barrier()
    launches = ptu.launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    value = ws * dofs / (ms / 1e3)

    # per-kernel event timings of a few more solves (graphs off): breakdown and roofline
    peaks, peak_src = load_peaks()
    tr = traffic_table()
    prof, ms_prof = kernel_profile(ptu, P, min(args.steps, 5), args.tol, args.max_it)
    roof = dominant_roofline(prof, prec == "fp64", dims, peaks, peak_src, tr)
    phases = {k: [r4(v["ms"] / min(args.steps, 5)), v["launches"] // min(args.steps, 5)]
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
    P.close()
    k2 = min(args.steps, 3)  # timed solves of the secondary entries (after one warm-up solve)

    extras = {}
    if not args.no_extras:
        # the Krylov-accelerated form (flexible GMRES(10) preconditioned by one Uzawa step), FP64
        Pk = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="fp64",
                         omega=args.omega, krylov=10)
        Pk.solve(args.tol, args.max_it)
        kms, kit = solve_timed(Pk, k2, args.tol, args.max_it)
        uk = np.zeros((prob.N, prob.ns))
        Pk.solve(args.tol, args.max_it, u_out=uk)
        Pk.close()
        extras["krylov"] = compact({"solver": "FGMRES(10), right preconditioner: one inexact Uzawa step",
                                    "value": dofs / (kms / 1e3), "ms_per_solve": kms, "iterations": kit,
                                    "rel_l2_vs_uzawa_solution": rel_l2(uk, u64)})
        # quasi-uniform random time steps (ratio <= 1.5, eq. 2.1-2.2), FP64
        taus = S.random_steps(prob.N, prob.T, 1, 0.5)
        Pn = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="fp64", taus=taus)
        Pn.solve(args.tol, args.max_it)
        nms, nit = solve_timed(Pn, k2, args.tol, args.max_it)
        Pn.close()
        extras["nonuniform_steps"] = compact({
            "steps": "tau_n = T w_n / sum w, w_n = 1 + 0.5 U_n (SplitMix64 seed 1), max/min %.3f"
                     % (taus.max() / taus.min()),
            "omega": "1.5 / (1 + alpha), alpha of eq. 2.2 with the step ratios",
            "value": dofs / (nms / 1e3), "ms_per_solve": nms, "iterations": nit})

    # the CPU leg of the headline workload (oracle on its first steps, in a fresh process)
    cpu = None
    rel64 = None
    ref2 = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        res2, ref2 = cpu_leg("heat2d%dx%d" % (args.n, args.nt) if wl == "heat2d" else wl, args.cpu_seconds,
                             64 if prob.dim < 3 else 1, single_thread=prob.dim < 3)
        cpu = cpu_baseline_entry(res2, prob)
        if ref2 is not None:
            rel64 = rel_l2(u64[:ref2.shape[0]], ref2)

    tail = {}
    if not args.no_extras and rank == 0:
        # the multigrid-only form: two V-cycles per H_k solve instead of the transform solves
        Pv = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="fp64", omega=args.omega,
                         h_solver="vcycle")
        Pv.solve(args.tol, args.max_it)
        vms, vit = solve_timed(Pv, k2, args.tol, args.max_it)
        vprof, _ = kernel_profile(ptu, Pv, 1, args.tol, args.max_it)
        uv = np.zeros((prob.N, prob.ns))
        Pv.solve(args.tol, args.max_it, u_out=uv)
        Pv.close()
        tail["vcycle_h"] = secondary(dofs / (vms / 1e3), vms, vit,
                                     rel_l2(uv[:ref2.shape[0]], ref2) if ref2 is not None else None,
                                     ref2.shape[0] if ref2 is not None else None,
                                     dominant_roofline(vprof, True, dims, peaks, peak_src, tr, short=True),
                                     precision="fp64")
        del uv

        # config 1: 1-D, 63 points, 64 steps, exact tridiagonal solves, FP64
        p1 = workload_problem("heat1d")
        P1 = ptu.Problem(p1.dim, p1.n, p1.N, p1.T, p1.coeff, S.source(p1), S.initial(p1), precision="fp64",
                         omega=args.omega, solver="exact")
        for _ in range(3):
            P1.solve(args.tol, args.max_it)
        ms1, it1 = solve_timed(P1, 20, args.tol, args.max_it)
        u1 = np.zeros((p1.N, p1.ns))
        P1.solve(args.tol, args.max_it, u_out=u1)
        P1.close()
        r1, ref1 = cpu_leg("heat1d", 5.0, p1.N) if not args.no_cpu else (None, None)
        tail["heat1d"] = secondary(p1.dofs / (ms1 / 1e3), ms1, it1,
                                   rel_l2(u1[:ref1.shape[0]], ref1) if ref1 is not None else None,
                                   ref1.shape[0] if ref1 is not None else None, None, precision="fp64",
                                   cpu_dofs_per_s=r1["value"] if r1 else None)

        # reduced batch (config 4 distribution, problems 0..B-1), mixed, one pt_solve_batch
        nb = args.batch_sample
        if nb > 0:
            bprobs = [S.batch_problem(i) for i in range(nb)]
            small = sorted(bprobs, key=lambda q: q.dofs)[:4]
            Ps = [make_batch_problem(ptu, q) for q in small]
            ptu.solve_batch(Ps, args.tol, args.max_it)
            for Q in Ps:
                Q.close()
            Ps = [make_batch_problem(ptu, q) for q in bprobs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bits, bsts = ptu.solve_batch(Ps, args.tol, args.max_it)
            torch.cuda.synchronize()
            bsec = time.perf_counter() - t0
            # the parity sample: the largest problem of the batch, against the oracle's first steps
            js = max(range(nb), key=lambda i: bprobs[i].dofs)
            us = np.zeros((bprobs[js].N, bprobs[js].ns))
            Ps[js].get_state(u_out=us)
            for Q in Ps:
                Q.close()
            rb, refb = cpu_leg("batch%d" % js, 8.0, 256) if not args.no_cpu else (None, None)
            tail["batch"] = secondary(sum(q.dofs for q in bprobs) / bsec, 1e3 * bsec, float(np.mean(bits)),
                                      rel_l2(us[:refb.shape[0]], refb) if refb is not None else None,
                                      refb.shape[0] if refb is not None else None, None, precision="mixed",
                                      problems=nb, iterations_max=int(max(bits)),
                                      converged=int(sum(1 for x in bsts if x == 0)),
                                      sample="problem %d (%dx%d, N_t %d)" % (js, bprobs[js].n[0], bprobs[js].n[1],
                                                                              bprobs[js].N))

        # config 3: 3-D 127^3 x 256, mixed precision (FP32 preconditioner, FP64 refinement)
        if not args.no_3d:
            p3 = workload_problem("heat3d")
            f3 = S.source(p3)
            P3 = ptu.Problem(p3.dim, p3.n, p3.N, p3.T, p3.coeff, f3, S.initial(p3), precision="mixed",
                             omega=args.omega)
            del f3
            P3.solve(args.tol, args.max_it)
            ms3, it3 = solve_timed(P3, k2, args.tol, args.max_it)
            prof3, _ = kernel_profile(ptu, P3, 1, args.tol, args.max_it)
            u3 = np.zeros((p3.N, p3.ns))
            P3.solve(args.tol, args.max_it, u_out=u3)
            P3.close()
            u3 = u3[:4].copy()
            r3, ref3 = cpu_leg("heat3d", 1.0, 1) if not args.no_cpu else (None, None)
            tail["heat3d"] = secondary(p3.dofs / (ms3 / 1e3), ms3, it3,
                                       rel_l2(u3[:ref3.shape[0]], ref3) if ref3 is not None else None,
                                       ref3.shape[0] if ref3 is not None else None,
                                       dominant_roofline(prof3, False, (3, p3.n[0], p3.N), peaks, peak_src, tr,
                                                         short=True),
                                       precision="mixed", cpu_dofs_per_s=r3["value"] if r3 else None)

    # config 2 in mixed precision (FP32 preconditioner and sweeps, FP64 refinement): the last key
    if not args.no_mixed:
        Pm = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, precision="mixed", omega=args.omega)
        Pm.solve(args.tol, args.max_it)
        barrier()
        mms, mit = solve_timed(Pm, min(args.steps, 10), args.tol, args.max_it)
        mms = max_over_ranks(mms, dist)
        mprof, _ = kernel_profile(ptu, Pm, 1, args.tol, args.max_it)
        um = np.zeros((prob.N, prob.ns))
        Pm.solve(args.tol, args.max_it, u_out=um)
        Pm.close()
        tail["mixed"] = secondary(ws * dofs / (mms / 1e3), mms, mit,
                                  rel_l2(um[:ref2.shape[0]], ref2) if ref2 is not None else None,
                                  ref2.shape[0] if ref2 is not None else None,
                                  dominant_roofline(mprof, False, dims, peaks, peak_src, tr, short=True),
                                  precision="mixed", rel_l2_vs_fp64_path=rel_l2(um, u64),
                                  speedup_vs_fp64=ms / mms,
                                  kernels={k: r4(v["ms"]) for k, v in
                                           sorted(mprof.items(), key=lambda kv: -kv[1]["ms"])[:8]})

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": dict(headline_config(prob, args.tol, args.omega, ws, prec, solver), iterations=iters),
            "gpu_launches": int(launches), "clocks": clk,
            "ms_per_step_with_kernel_events": ms_prof,
            "kernels_ms_launches_per_solve": phases,
            "path_roofline": compact(path_roofline(prof, dims, iters, value, prec, peaks, min(args.steps, 5))),
            **extras,
            "e2e": e2e, "cpu_baseline": compact(cpu), "rel_l2_vs_oracle": r4(rel64),
            "oracle_steps": None if ref2 is None else int(ref2.shape[0]), "roofline": roof,
            **tail,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
