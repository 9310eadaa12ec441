"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element."""
import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import mg
from oracle import spacetime as st

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10      # relative L2 vs the oracle for FP64 solves
MIXED_TOL = 1e-8      # relative L2 vs the oracle after refinement, mixed precision


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1802_08126_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def make(prob, precision="fp64", solver="mg", omega=0.5):
    import paper_1802_08126_gb300 as ptu
    return ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), S.initial(prob),
                       precision=precision, solver=solver, omega=omega)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SMALL = [S.heat1d_mms(15, 16), S.heat2d_uniform(15, 8), S.heat2d_uniform(31, 4),
         S.heat3d_bumps(7, 4), S.heat2d_uniform(3, 1), S.heat1d_mms(1, 2)]
# N not a power of two (Bluestein path of the temporal transform), including primes
GENERAL_N = [S.heat2d_uniform(7, 3), S.heat2d_uniform(15, 12), S.heat1d_mms(15, 97),
             S.heat2d_uniform(7, 1000), S.heat1d_mms(7, 2047)]


@pytest.mark.parametrize("prob", GENERAL_N, ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dst_general_N_matches_sine_sums(prob, precision):
    tol = 1e-12 if precision == "fp64" else 2e-6
    rng = np.random.default_rng(7)
    r = rng.standard_normal((prob.N, prob.ns))
    with make(prob, precision) as P:
        out = torch.empty_like(dev(r))
        P.dst_forward(dev(r), out)
        ref = st.dst_forward(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * np.log2(2 * prob.N)
        P.dst_inverse(dev(r), out)
        ref = st.dst_inverse(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * np.log2(2 * prob.N)


# power-of-two N of the CTA-cooperative radix-8 Stockham kernels (several passes, the sizes of
# the 2-D and batch workloads), against the sine sums of §4 computed densely by the oracle
POW2_N = [S.heat2d_uniform(15, 256), S.heat2d_uniform(31, 1024), S.heat1d_mms(15, 2048), S.heat2d_uniform(7, 512)]


@pytest.mark.parametrize("prob", POW2_N, ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dst_power_of_two_N_matches_sine_sums(prob, precision):
    tol = 1e-12 if precision == "fp64" else 2e-6
    rng = np.random.default_rng(17)
    r = rng.standard_normal((prob.N, prob.ns))
    with make(prob, precision) as P:
        out = torch.empty_like(dev(r))
        P.dst_forward(dev(r), out)
        ref = st.dst_forward(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * np.log2(prob.N)
        P.dst_inverse(dev(r), out)
        ref = st.dst_inverse(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * np.log2(prob.N)


@pytest.mark.parametrize("prob", [S.heat2d_uniform(15, 24), S.heat1d_mms(31, 37)], ids=lambda p: p.name)
def test_general_N_solve_matches_oracle(prob):
    f, u0 = S.source(prob), S.initial(prob)
    with make(prob, omega=0.5) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 1000, u_out=u)
    assert stt == 0
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0)
    assert rel_err(u, ref) <= FP64_TOL


@pytest.mark.parametrize("prob", SMALL, ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dst_both_directions_match_sine_sums(prob, precision):
    tol = 1e-12 if precision == "fp64" else 2e-6
    rng = np.random.default_rng(3)
    r = rng.standard_normal((prob.N, prob.ns))
    with make(prob, precision) as P:
        out = torch.empty_like(dev(r))
        P.dst_forward(dev(r), out)
        ref = st.dst_forward(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * max(1, np.log2(prob.N))
        P.dst_inverse(dev(r), out)
        ref = st.dst_inverse(r)
        assert np.abs(host(out) - ref).max() <= tol * np.abs(ref).max() * max(1, np.log2(prob.N))


@pytest.mark.parametrize("prob", SMALL, ids=lambda p: p.name)
def test_apply_B_matches_oracle(prob):
    rng = np.random.default_rng(4)
    u = rng.standard_normal((prob.N, prob.ns))
    with make(prob) as P:
        out = torch.empty_like(dev(u))
        P.apply_B(dev(u), out)
    ref = oracle.apply_B(prob.dim, prob.n, prob.N, prob.T, prob.coeff, u)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()


# 63^2 and 127^2 reach the warp-strip level kernels (fine levels of width >= 64), 255^2 and 511^2
# wider 2-D levels; 15^3, 31^3 and 63^3 the 3-D levels run by the level kernels (slices above 1024
# points: one, two and three levels) before the one-CTA coarse kernel
@pytest.mark.parametrize("prob", SMALL[:4] + [S.heat2d_uniform(63, 3), S.heat2d_uniform(127, 2),
                                              S.heat2d_uniform(255, 3), S.heat2d_uniform(511, 2),
                                              S.heat3d_bumps(15, 3), S.heat3d_bumps(31, 2), S.heat3d_bumps(63, 2),
                                              S.heat1d_mms(2047, 2)],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cycles", [1, 2, 3])
def test_vcycle_preconditioners_match_oracle_vcycle(prob, precision, cycles):
    # FP64: summation orders differ, the difference grows with the condition number of the level
    # operators, ~4/(pi h)^2 (1.7e6 for the 1-D grid of 2047 points)
    kappa = 4.0 / (np.pi / (prob.n[0] + 1)) ** 2
    tol = max(1e-11, kappa * 1e-16) if precision == "fp64" else 5e-6
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    Asolve, Hsolve = mg.st_vcycles(T, h_cycles=cycles)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((prob.N, prob.ns))
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), S.initial(prob),
                     precision=precision, omega=0.5, n_vcycles=cycles, h_solver="vcycle") as P:
        out = torch.empty_like(dev(r))
        P.precond_A(dev(r), out)
        ref = Asolve(r)
        assert rel_err(host(out), ref) <= tol
        P.precond_H(dev(r), out)
        ref = T.apply_Hinv(r, Hsolve)
        assert rel_err(host(out), ref) <= tol


@pytest.mark.parametrize("prob", [S.heat2d_uniform(15, 8), S.heat2d_uniform(31, 12), S.heat2d_uniform(7, 2),
                                  S.heat2d_uniform(63, 5), S.heat2d_uniform(1, 4), S.heat2d_uniform(3, 3),
                                  S.heat2d_uniform(127, 2), S.heat2d_uniform(255, 2), S.heat3d_bumps(7, 4),
                                  S.heat3d_bumps(15, 3), S.heat3d_bumps(31, 2)], ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_exact_transform_H_matches_oracle_direct_solves(prob, precision):
    """H~^-1 with exact H_k solves done by spatial sine transforms equals Phi^-1 Hhat^-1 Phi^-T
    with sparse direct H_k solves (§4, eq. 4.4)."""
    tol = 1e-11 if precision == "fp64" else 5e-6
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    rng = np.random.default_rng(9)
    r = rng.standard_normal((prob.N, prob.ns))
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), None, precision=precision,
                     h_solver="exact") as P:
        out = torch.empty_like(dev(r))
        P.precond_H(dev(r), out)
    assert rel_err(host(out), T.apply_Hinv(r, T.exact_H_solver())) <= tol


# 3-D grids whose xy planes fit in one CTA (n + 1 = 64, 128: the whole-plane x and y transforms
# around the z pass) and a 2-D grid of the whole-plane block solve, against H_k solves by the
# sine-transform solver (pinned to the sparse direct solves in tests/test_oracle_spectral.py;
# the direct solves are too slow at these sizes)
@pytest.mark.parametrize("prob", [S.heat3d_bumps(63, 2), S.heat3d_bumps(127, 2), S.heat2d_uniform(127, 6)],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_exact_transform_H_large_grids_match_sine_solves(prob, precision):
    from tests.conftest import sine_H_solver
    tol = 1e-11 if precision == "fp64" else 5e-6
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    rng = np.random.default_rng(19)
    r = rng.standard_normal((prob.N, prob.ns))
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), None, precision=precision,
                     h_solver="exact") as P:
        out = torch.empty_like(dev(r))
        P.precond_H(dev(r), out)
    assert rel_err(host(out), T.apply_Hinv(r, sine_H_solver(T))) <= tol


# n + 1 <= 1024: parallel cyclic reduction; 2047: the sequential elimination
@pytest.mark.parametrize("prob,precision", [(S.heat1d_mms(63, 64), "fp64"), (S.heat1d_mms(63, 64), "mixed"),
                                            (S.heat1d_mms(1, 4), "fp64"), (S.heat1d_mms(1, 4), "mixed"),
                                            (S.heat1d_mms(15, 5), "fp64"), (S.heat1d_mms(1023, 6), "fp64"),
                                            (S.heat1d_mms(2047, 3), "fp64")], ids=lambda v: getattr(v, "name", v))
def test_exact_1d_preconditioners_match_oracle(prob, precision):
    # Elimination in precision eps: relative error up to ~kappa * eps with kappa(tau A_n) ~
    # 4/(pi h)^2 (1.7e3 at h = 1/64): FP32 ~1e-4; FP64 1e-12 up to h = 1/64, kappa * 1e-15 beyond.
    kappa = 4.0 / (np.pi / (prob.n[0] + 1)) ** 2
    tol = max(1e-12, kappa * 1e-15) if precision == "fp64" else 1e-4
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    rng = np.random.default_rng(6)
    r = rng.standard_normal((prob.N, prob.ns))
    with make(prob, precision, solver="exact") as P:
        out = torch.empty_like(dev(r))
        P.precond_A(dev(r), out)
        assert rel_err(host(out), T.exact_A_solver()(r)) <= tol
        P.precond_H(dev(r), out)
        assert rel_err(host(out), T.apply_Hinv(r, T.exact_H_solver())) <= tol


def test_heat1d_exact_solves_matches_oracle_and_mirror_history():
    """The 1-D manufactured problem with exact spatial solves: the GPU residual history
    follows the oracle's Uzawa iteration (eq. 3.1) step by step, and the converged u is the
    implicit-Euler solution."""
    prob = S.heat1d_mms(63, 64)
    f, u0 = S.source(prob), S.initial(prob)
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    F = T.rhs(f, u0)
    _, _, hist_ref = T.uzawa(F, 0.5, 25, T.exact_A_solver(), T.exact_H_solver())
    with make(prob, solver="exact", omega=0.5) as P:
        stt, it, hist = P.solve(0.0, 25)
        assert it == 25
        assert np.abs(hist - hist_ref).max() <= 1e-10 * hist_ref.max()
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-13, 400, u_out=u)
    assert stt == 0
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0)
    assert rel_err(u, ref) <= FP64_TOL


@pytest.mark.parametrize("prob", [S.heat2d_uniform(31, 32), S.heat3d_bumps(7, 16), S.heat1d_mms(31, 16)],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("hsol", ["vcycle", "exact"])
def test_multigrid_solve_history_and_solution(prob, hsol):
    if hsol == "exact" and prob.dim == 1:
        pytest.skip("transform H_k solves are 2-D and 3-D (1-D has its own exact solves)")
    f, u0 = S.source(prob), S.initial(prob)
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    F = T.rhs(f, u0)
    Asolve, Hsolve = mg.st_vcycles(T)
    if hsol == "exact":
        Hsolve = T.exact_H_solver()
    _, _, hist_ref = T.uzawa(F, 0.5, 15, Asolve, lambda k, r: Hsolve(k, r))
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, omega=0.5, h_solver=hsol) as P:
        _, it, hist = P.solve(0.0, 15)
        assert np.abs(hist - hist_ref).max() <= 1e-9 * hist_ref.max()
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 1000, u_out=u)
    assert stt == 0
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0)
    assert rel_err(u, ref) <= FP64_TOL


# 31^3 and 63^3 take the row-streamed 3-D FP32 step (bands of 8 and 4 rows), 255^2 and 511^2 the
# row-streamed 2-D step (one and two 256-column segments per row)
@pytest.mark.parametrize("prob", [S.heat2d_uniform(31, 32), S.heat3d_bumps(7, 16), S.heat3d_bumps(31, 8),
                                  S.heat3d_bumps(63, 4), S.heat2d_uniform(255, 6), S.heat2d_uniform(511, 3)],
                         ids=lambda p: p.name)
def test_mixed_precision_refines_to_fp64_solution(prob):
    f, u0 = S.source(prob), S.initial(prob)
    with make(prob, precision="mixed", omega=0.5) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-11, 1000, u_out=u)
    assert stt == 0
    # (3-D above 31^3: the oracle's CG stepping, the banded factor being too wide)
    method = "cg" if prob.dim == 3 and prob.n[0] > 31 else "cholesky"
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, method=method)
    assert rel_err(u, ref) <= MIXED_TOL
    # the residual the library reports is the residual of the u it returns (the Dirichlet
    # ghosts of the device layout stayed exactly zero)
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    assert abs(T.residual(T.rhs(f, u0), u) - hist[-1]) <= 0.01 * hist[-1] + 1e-15


def test_not_converged_still_returns_iterate():
    prob = S.heat2d_uniform(15, 8)
    with make(prob) as P:
        u = np.full((prob.N, prob.ns), np.nan)
        stt, it, hist = P.solve(1e-14, 3, u_out=u)
    from paper_1802_08126_gb300 import PT_ENOTCONV
    assert stt == PT_ENOTCONV and it == 3 and len(hist) == 4
    assert np.isfinite(u).all() and hist[0] == pytest.approx(1.0)


def test_device_buffers_round_trip():
    """f given on the device and u returned to the device give the same answer as host buffers."""
    prob = S.heat2d_uniform(15, 8)
    import paper_1802_08126_gb300 as ptu
    f = S.source(prob)
    P = ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, dev(f), None)
    ud = torch.zeros((prob.N, prob.ns), dtype=torch.float64, device="cuda")
    P.solve(1e-12, 500, u_out=ud)
    uh = np.zeros((prob.N, prob.ns))
    P.set_rhs(f)
    P.solve(1e-12, 500, u_out=uh)
    P.close()
    assert np.array_equal(host(ud), uh)


@pytest.mark.parametrize("prob", [S.heat2d_uniform(31, 32), S.heat2d_uniform(63, 64), S.heat3d_bumps(15, 16),
                                  S.heat1d_mms(31, 40)], ids=lambda p: p.name)
def test_krylov_accelerated_solve_matches_oracle(prob):
    """Flexible GMRES(20) preconditioned by one Uzawa step (§8.3's acceleration): the same solution
    as the oracle's implicit Euler, in fewer iterations than the plain Uzawa iteration."""
    import paper_1802_08126_gb300 as ptu
    f, u0 = S.source(prob), S.initial(prob)
    solver = "exact" if prob.dim == 1 else "mg"
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, omega=0.5, solver=solver) as P:
        _, it_plain, _ = P.solve(1e-12, 1000)
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, omega=0.5, solver=solver,
                     krylov=20) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 1000, u_out=u)
    assert stt == 0
    assert it < it_plain, (it, it_plain)
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0)
    assert rel_err(u, ref) <= FP64_TOL
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    assert abs(T.residual(T.rhs(f, u0), u) - hist[-1]) <= 0.01 * hist[-1] + 1e-15
