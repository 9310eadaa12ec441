"""Parity of the CUDA path with the oracle on non-uniform time steps tau_n (§2, eq. 2.1-2.2):
B = K + diag(tau_n A_n), F_n = tau_n f_n, the preconditioner on the reference pair (T/N, Abar)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import mg
from oracle import spacetime as st

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-8
OMEGA = 0.45   # inside the convergence range of the spread-0.5 step families below


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1802_08126_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def steps(p, seed=17, spread=0.5):
    return dataclasses.replace(p, taus=S.random_steps(p.N, p.T, seed, spread))


def const_coeff(p):
    """The same problem with a = a0 (constant): the reference coefficient is constant, so the
    2-D/3-D H_k solves take the exact spatial-transform path whatever the steps."""
    return dataclasses.replace(p, coeff=S.Coeff(p.coeff.a0, 0.0))


def problem(p, **kw):
    import paper_1802_08126_gb300 as ptu
    kw.setdefault("omega", OMEGA)
    return ptu.Problem(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), S.initial(p), taus=p.taus, **kw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def stepping(p, **kw):
    return oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), S.initial(p), taus=p.taus, **kw)


SMALL = [steps(S.heat1d_mms(15, 16)), steps(S.heat2d_uniform(15, 8)), steps(S.heat2d_uniform(31, 4)),
         steps(S.heat3d_bumps(7, 4)), steps(S.heat2d_uniform(3, 1)), steps(S.heat2d_uniform(7, 12))]


@pytest.mark.parametrize("prob", SMALL, ids=lambda p: p.name)
def test_apply_B_matches_oracle(prob):
    u = np.random.default_rng(4).standard_normal((prob.N, prob.ns))
    with problem(prob) as P:
        out = torch.empty_like(dev(u))
        P.apply_B(dev(u), out)
    ref = oracle.apply_B(prob.dim, prob.n, prob.N, prob.T, prob.coeff, u, taus=prob.taus)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prob", SMALL[:4] + [steps(S.heat2d_uniform(63, 3)), steps(S.heat2d_uniform(127, 2))],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_A_solver_is_the_vcycle_of_tau_n_A_n(prob, precision):
    """The library forms its V-cycles for tau A_n and scales by rho_n = tau / tau_n; the oracle
    builds the V-cycle of tau_n A_n itself: the two agree (the V-cycle is homogeneous of degree -1
    in the operator)."""
    tol = 1e-11 if precision == "fp64" else 5e-6
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, taus=prob.taus)
    Asolve, _ = mg.st_vcycles(T)
    r = np.random.default_rng(5).standard_normal((prob.N, prob.ns))
    with problem(prob, precision=precision) as P:
        out = torch.empty_like(dev(r))
        P.precond_A(dev(r), out)
        assert rel_err(host(out), Asolve(r)) <= tol


@pytest.mark.parametrize("prob", [steps(S.heat2d_uniform(31, 32)), steps(S.heat2d_uniform(15, 8)),
                                  steps(S.heat3d_bumps(7, 16)), steps(S.heat1d_mms(31, 16)),
                                  steps(S.heat2d_uniform(63, 24)), const_coeff(steps(S.heat2d_uniform(31, 16))),
                                  const_coeff(steps(S.heat3d_bumps(15, 8))), steps(S.heat3d_bumps(15, 8))],
                         ids=lambda p: p.name)
@pytest.mark.parametrize("hsol", ["vcycle", "exact"])
def test_history_follows_oracle_and_solution(prob, hsol):
    """The residual history follows the oracle's Uzawa iteration (eq. 3.1) with tau_n A_n in B and
    in the A~ V-cycles, and the converged u is the implicit-Euler solution on the same steps.  The
    reference coefficient (the time mean) of these periodic coefficients is constant, so the
    exact transform H_k solves apply on any time grid."""
    if hsol == "exact" and prob.dim == 1:
        pytest.skip("transform H_k solves are 2-D and 3-D")
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, taus=prob.taus)
    F = T.rhs(S.source(prob), S.initial(prob))
    Asolve, Hsolve = mg.st_vcycles(T)
    if hsol == "exact":
        Hsolve = T.exact_H_solver()
    _, _, hist_ref = T.uzawa(F, OMEGA, 15, Asolve, lambda k, r: Hsolve(k, r))
    with problem(prob, h_solver=hsol) as P:
        _, it, hist = P.solve(0.0, 15)
        assert it == 15
        assert np.abs(hist - hist_ref).max() <= 1e-9 * hist_ref.max()
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 2000, u_out=u)
    assert stt == 0
    assert rel_err(u, stepping(prob)) <= FP64_TOL


def test_exact_1d_solves_follow_oracle():
    prob = steps(S.heat1d_mms(63, 64), seed=3)
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, taus=prob.taus)
    F = T.rhs(S.source(prob), S.initial(prob))
    _, _, hist_ref = T.uzawa(F, OMEGA, 25, T.exact_A_solver(), T.exact_H_solver())
    with problem(prob, solver="exact") as P:
        _, it, hist = P.solve(0.0, 25)
        assert np.abs(hist - hist_ref).max() <= 1e-10 * hist_ref.max()
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-13, 1000, u_out=u)
    assert stt == 0
    assert rel_err(u, stepping(prob)) <= FP64_TOL
    # the manufactured solution on the same steps: first order in max tau
    assert np.abs(u - S.mms1_exact(63, 64, prob.T, prob.taus)).max() < 2e-3


# 31^3 takes the 3-D strip kernels of the refinement, 31^2 the 2-D ones, 7^3 the generic ones
@pytest.mark.parametrize("prob", [steps(S.heat2d_uniform(31, 32)), steps(S.heat3d_bumps(31, 8)),
                                  steps(S.heat3d_bumps(7, 16)), steps(S.heat2d_uniform(15, 8)),
                                  const_coeff(steps(S.heat2d_uniform(63, 16))), steps(S.heat2d_uniform(255, 6))],
                         ids=lambda p: p.name)
def test_mixed_precision_refines_to_fp64_solution(prob):
    with problem(prob, precision="mixed") as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-11, 2000, u_out=u)
    assert stt == 0
    assert rel_err(u, stepping(prob)) <= MIXED_TOL
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, taus=prob.taus)
    assert abs(T.residual(T.rhs(S.source(prob), S.initial(prob)), u) - hist[-1]) <= 0.01 * hist[-1] + 1e-15


@pytest.mark.parametrize("prob", [steps(S.heat2d_uniform(31, 32)), steps(S.heat3d_bumps(15, 16)),
                                  steps(S.heat1d_mms(31, 40))], ids=lambda p: p.name)
def test_krylov_accelerated_solve_matches_oracle(prob):
    solver = "exact" if prob.dim == 1 else "mg"
    with problem(prob, solver=solver) as P:
        _, it_plain, _ = P.solve(1e-12, 2000)
    with problem(prob, solver=solver, krylov=20) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 2000, u_out=u)
    assert stt == 0
    assert it < it_plain, (it, it_plain)
    assert rel_err(u, stepping(prob)) <= FP64_TOL


def test_equal_steps_give_the_uniform_results_bitwise():
    """Passing T/N for every step is the uniform problem: identical iterates and solution."""
    prob = S.heat2d_uniform(31, 16)
    same = dataclasses.replace(prob, taus=np.full(prob.N, prob.T / prob.N))
    out = []
    for p in (prob, same):
        with problem(p, omega=0.5) as P:
            u = np.zeros((p.N, p.ns))
            _, it, hist = P.solve(1e-12, 1000, u_out=u)
        out.append((u, hist))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_server_copies_the_steps():
    """A queued request keeps its own copy of the step lengths; the result is the solo solve's."""
    import paper_1802_08126_gb300 as ptu
    prob = steps(S.heat2d_uniform(31, 16), seed=5)
    f = S.source(prob)
    with problem(prob) as P:
        u_solo = np.zeros((prob.N, prob.ns))
        P.solve(1e-10, 1000, u_out=u_solo)
    sv = ptu.Server()
    try:
        taus = prob.taus.copy()
        t = sv.submit(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f=f, tol=1e-10, max_it=1000,
                      taus=taus, precision="fp64", omega=OMEGA)
        taus[:] = np.nan   # the caller's array changes after the submission
        u = np.zeros((prob.N, prob.ns))
        stt, it = sv.wait(t, u_out=u)
    finally:
        sv.close()
    assert stt == 0
    assert np.array_equal(u, u_solo)


def test_full_size_heat2d_random_steps_first_steps_and_global_residual():
    """The 2-D workload at full size (255^2 grid, 1024 random steps with ratio <= 1.5, FP64):
    the first steps against the oracle's implicit Euler on the same steps, and the residual of
    the returned u recomputed with the oracle's B."""
    prob = steps(S.heat2d_uniform(255, 1024), seed=1)
    f = S.source(prob)
    with problem(prob) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 3000, u_out=u)
    assert stt == 0
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None, steps=3, taus=prob.taus)
    assert rel_err(u[:3], ref) <= FP64_TOL
    F = prob.taus[:, None] * f
    Bu = oracle.apply_B(prob.dim, prob.n, prob.N, prob.T, prob.coeff, u, taus=prob.taus)
    assert np.linalg.norm(F - Bu) / np.linalg.norm(F) <= 1e-12 * 1.01


@pytest.mark.parametrize("prob", [S.heat2d_uniform(31, 16), steps(S.heat2d_uniform(31, 16), seed=2),
                                  steps(S.heat3d_bumps(15, 6), seed=6), steps(S.heat1d_mms(31, 12), seed=7)],
                         ids=lambda p: p.name + ("_uniform" if p.taus is None else "_steps"))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_buffers_match_device_buffers(prob, precision):
    """Host f and u move through the work buffer in chunks of whole slices (two or more chunks in
    mixed precision here): the same F, iterates and u as with device buffers, bit for bit."""
    import paper_1802_08126_gb300 as ptu
    f, u0 = S.source(prob), S.initial(prob)
    out = []
    for on_dev in (False, True):
        fa = dev(f) if on_dev else f
        with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, fa, u0, precision=precision,
                         omega=OMEGA, taus=prob.taus) as P:
            if on_dev:
                u = torch.zeros((prob.N, prob.ns), dtype=torch.float64, device="cuda")
                _, it, hist = P.solve(1e-10, 1000, u_out=u)
                u = host(u)
            else:
                u = np.zeros((prob.N, prob.ns))
                _, it, hist = P.solve(1e-10, 1000, u_out=u)
        out.append((u, hist))
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])
