"""Host-side arithmetic of the benchmark's roofline entries (no GPU)."""
import math

import numpy as np
import pytest

import bench

PEAKS = {"hbm_gbs": 6696.2, "sm_max_mhz": 2070.0}


def test_path_roofline_bounds_and_fraction():
    n, N, its, steps = 255, 1024, 53, 3
    # per-solve launch counts of the FP64 2-D iteration, summed over `steps` solves
    per_it = {"dsti_rows": 2, "dst_forward": 1, "dst_inverse": 1, "hsolve_y": 1, "resid_bres": 1,
              "mg2_up": 3, "mg2_down": 3, "resid_u_bres": 1}
    prof = {k: {"launches": c * its * steps, "ms": 1.0, "bytes": 1.0} for k, c in per_it.items()}
    out = bench.path_roofline(prof, (2, n, N), its, 5.9e7, "fp64", PEAKS, steps)
    dofs = float(N) * n * n
    assert out["hbm_bound_dofs_per_s"] == pytest.approx(6696.2e9 / (368.0 * its))
    fl = sum(bench.fp64_flops_per_launch(k, 2, n, N) * c * its for k, c in per_it.items()
             if bench.fp64_flops_per_launch(k, 2, n, N) is not None)
    peak = 152 * 2 * 2 * 2070e6
    assert out["fp64_bound_dofs_per_s"] == pytest.approx(peak * dofs / fl)
    assert out["fp64_flops_per_dof_iteration"] == pytest.approx(fl / dofs / its)
    bound = min(out["hbm_bound_dofs_per_s"], out["fp64_bound_dofs_per_s"])
    assert out["frac"] == pytest.approx(5.9e7 / bound)
    assert out["bound"] == ("hbm" if bound == out["hbm_bound_dofs_per_s"] else "fp64")
    # the DST-I count: a real FFT of length n + 1 per line, 2.5 M log2 M
    assert bench.fp64_flops_per_launch("dsti_rows", 2, n, N) == pytest.approx(N * n * 2.5 * 256 * math.log2(256))


def test_path_roofline_mixed_and_unmodelled():
    out = bench.path_roofline({}, (2, 255, 1024), 53, 2.9e8, "mixed", PEAKS, 3)
    assert out["bound"] == "hbm" and "fp64_bound_dofs_per_s" not in out
    assert out["frac"] == pytest.approx(2.9e8 / (6696.2e9 / (232.0 * 53)))
    assert bench.path_roofline({}, (1, 63, 64), 60, 7.6e5, "fp64", PEAKS, 3) is None
    assert bench.path_roofline({}, (2, 255, 1024), 53, 1.0, "mixed", {}, 3) is None  # no peaks


def test_cpu_leg_runs_the_oracle_in_a_fresh_process():
    """The CPU leg returns the oracle's first steps of the named workload and its timing (all
    cores, and one thread on the first step)."""
    import oracle
    import synthetic as S
    res, u = bench.cpu_leg("heat2d31x8", 0.5, 4, single_thread=True)
    assert res is not None and res["cores"] >= 1 and res["value"] > 0
    assert res["single_thread"]["cores"] == 1 and res["single_thread"]["value"] > 0
    k = res["k"]
    assert 1 <= k <= 4 and u.shape == (k, 31 * 31)
    p = S.heat2d_uniform(31, 8)
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p, steps=k), None, steps=k)
    assert np.array_equal(u, ref)


def test_workload_names_and_rounding():
    assert bench.workload_problem("heat2d").n == [255, 255]
    assert bench.workload_problem("heat2d63x32").N == 32
    assert bench.workload_problem("heat3d").dim == 3
    assert bench.workload_problem("batch7").name == S_batch_name(7)
    assert bench.r4(123456.789) == 123500.0 and bench.r4(3) == 3 and bench.r4(None) is None
    assert bench.compact({"a": 1.23456789, "b": {"c": 2.0000001}, "d": "x"}) == {"a": 1.235, "b": {"c": 2.0}, "d": "x"}


def S_batch_name(i):
    import synthetic as S
    return S.batch_problem(i).name
