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
    t0 = time.perf_counter()
    oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, steps=1)
    one = time.perf_counter() - t0
    k = int(max(1, min(f.shape[0], seconds / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, steps=k)
    secs = time.perf_counter() - t0
    return k * prob.ns / secs, k, secs, cores


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


def main():
    args = parse()
    rank, ws, local, dist = dist_init(args)
    if args.impl == "reference":
        return run_reference(args, rank, ws, dist)

    import torch

    import paper_1802_08126_gb300 as ptu
    from paper_1802_08126_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prob = S.heat2d_uniform(args.n, args.nt)
    dofs = prob.dofs
    f = S.source(prob)
    P = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, precision="fp64",
                    omega=args.omega)

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
    ptu.profile_reset()
    ptu.profile_enable(True)
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
    ptu.profile_enable(False)
    prof = ptu.profile_totals()
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    value = ws * dofs * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (largest share of the timed region)
    peaks, peak_src = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roof = None
    if dom is not None:
        name, d = dom
        per_launch_ms = d["ms"] / max(d["launches"], 1)
        gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
        tr = traffic_table()
        traffic = tr.get((name, WORKLOAD))
        roof = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": traffic,
                "algorithmic_bytes_per_launch": d["bytes"] / max(d["launches"], 1),
                "avg_launch_ms": per_launch_ms, "share": d["ms"] / sum(v["ms"] for v in prof.values()),
                "peak_source": peak_src}
    phases = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                  "GBps": v["bytes"] / max(v["ms"], 1e-9) / 1e6}
              for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    # end to end through the C ABI: pinned host source in, solution out, every step
    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(f).pin_memory().numpy()
        uh = torch.empty((prob.N, prob.ns), dtype=torch.float64).pin_memory().numpy()
        P.set_rhs(fh)
        P.solve(args.tol, args.max_it, u_out=uh)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.set_rhs(fh)
            st, it, hist = P.solve(args.tol, args.max_it, u_out=uh)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        barrier()
        if dist is not None:
            t = torch.tensor([secs], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            secs = t.item()
        e2e = {"value": ws * dofs * args.steps / secs, "unit": "DOF/s",
               "h2d_bytes_per_step": int(fh.nbytes), "d2h_bytes_per_step": int(uh.nbytes + 8 * (it + 1))}
        u64 = uh.copy()
    else:
        u64 = np.zeros((prob.N, prob.ns))
        P.solve(args.tol, args.max_it, u_out=u64)

    # the mixed-precision form on the same workload
    mixed = None
    if not args.no_mixed:
        Pm = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, precision="mixed",
                         omega=args.omega)
        solve_once(Pm)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mits = []
        for _ in range(args.steps):
            it, res = solve_once(Pm)
            mits.append(it)
        e1.record()
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1)
        um = np.zeros((prob.N, prob.ns))
        Pm.solve(args.tol, args.max_it, u_out=um)
        Pm.close()
        if dist is not None:
            t = torch.tensor([mms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            mms = t.item()
        mixed = {"value": ws * dofs * args.steps / (mms / 1e3), "unit": "DOF/s",
                 "ms_per_step": mms / args.steps, "iterations": mits[-1],
                 "rel_l2_vs_fp64_path": float(np.linalg.norm(um - u64) / np.linalg.norm(u64))}
    P.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, k, secs, cores = cpu_sample(prob, args.cpu_seconds, f[:64])
        cpu = {"value": v, "unit": "DOF/s", "cores": cores, "kind": "oracle",
               "sample": "first %d of %d implicit-Euler steps, banded Cholesky per step (%.1f s)"
                         % (k, prob.N, secs)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [prob.n[0]] * 2, "N_t": prob.N, "T": prob.T,
                       "dofs_per_gpu": dofs, "tol": args.tol, "omega": args.omega,
                       "iterations": its[-1], "spatial_solver": "V(1,1) geometric multigrid",
                       "l2": "inputs larger than L2 (533 MB per space-time vector)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "mixed": mixed, "kernels": phases,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
