"""Pins of the oracle with non-uniform time steps tau_n (§2, eq. 2.1-2.2): closed forms, a
convergence order, brute-force dense solves and the agreement of its two independent
implementations (C stepping and NumPy/SciPy time-global operators).  No GPU."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import mg
from oracle import spacetime as st


def _with_steps(p, seed, spread=0.5):
    return dataclasses.replace(p, taus=S.random_steps(p.N, p.T, seed, spread))


@pytest.mark.parametrize("dim,n,mode,a0", [(1, 31, (3,), 0.7), (2, 15, (2, 5), 1.3), (3, 7, (1, 2, 3), 2.0)])
def test_eigenmode_decay_closed_form_nonuniform(dim, n, mode, a0):
    """Constant a: u_n = prod_{m <= n} (1 + tau_m lambda_h)^-1 u0 for the eigenvector
    u0 = prod sin(m_d pi x_d), lambda_h = sum_d 4 a0 h^-2 sin^2(m_d pi h / 2)."""
    p = _with_steps(S.eigenmode(dim, n, 12, 0.3, a0, mode), seed=11 + dim)
    u0 = S.initial(p)
    u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), u0, taus=p.taus)
    h = 1.0 / (n + 1)
    lam = sum(4 * a0 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2 for m in mode)
    g = np.cumprod(1.0 / (1.0 + p.taus * lam))
    exact = g[:, None] * u0[None, :]
    assert np.abs(u - exact).max() < 1e-13
    # a plausible slip (uniform steps) is far off
    g_uni = (1.0 + (p.T / p.N) * lam) ** -np.arange(1, p.N + 1)
    assert np.abs(g - g_uni).max() > 1e-3


def test_apply_B_nonuniform_closed_form_and_stepping():
    """(B u)_n = (g_n - g_{n-1}) phi + tau_n lambda g_n phi for u_n = g_n phi with an eigenvector
    phi of the constant-coefficient A; and B u = F for the stepped u of a variable coefficient."""
    p = _with_steps(S.eigenmode(2, 15, 9, 0.4, 1.1, (3, 2)), seed=5)
    phi = S.initial(p)
    h = 1.0 / 16
    lam = sum(4 * 1.1 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2 for m in (3, 2))
    g = np.linspace(1.0, -0.5, p.N) ** 3
    u = g[:, None] * phi[None, :]
    gm = np.concatenate([[0.0], g[:-1]])
    exact = ((g - gm) + p.taus * lam * g)[:, None] * phi[None, :]
    assert np.abs(oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, u, taus=p.taus) - exact).max() < 1e-11
    q = _with_steps(S.heat2d_uniform(7, 6), seed=9)
    f = S.source(q)
    uq = oracle.implicit_euler(q.dim, q.n, q.N, q.T, q.coeff, f, taus=q.taus)
    F = st.SpaceTime(q.dim, q.n, q.N, q.T, q.coeff, taus=q.taus).rhs(f, None)
    assert np.abs(oracle.apply_B(q.dim, q.n, q.N, q.T, q.coeff, uq, taus=q.taus) - F).max() < 1e-13


def test_c_and_numpy_operators_agree_nonuniform():
    """The C action of B and the SciPy-assembled time-global B (separate implementations)."""
    p = _with_steps(S.heat3d_bumps(5, 7), seed=21)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, taus=p.taus)
    v = np.random.default_rng(3).standard_normal((p.N, p.ns))
    a = oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, v, taus=p.taus)
    assert np.abs(a - T.B(v)).max() < 1e-11 * np.abs(a).max()


def test_mms_order_nonuniform():
    """Manufactured 1-D problem on random steps (spread 0.5): error O(max tau + h^2); refining
    h by 2 and the steps by 4 divides the max error by about 4."""
    errs = []
    for n, N, seed in [(63, 64, 1), (127, 256, 2)]:
        p = _with_steps(S.heat1d_mms(n, N), seed)
        u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), S.initial(p), taus=p.taus)
        errs.append(np.abs(u - S.mms1_exact(n, N, p.T, p.taus)).max())
    assert 1e-4 < errs[0] < 2e-3
    assert 3.3 < errs[0] / errs[1] < 4.7


@pytest.mark.parametrize("prob", [S.heat1d_mms(7, 8), S.heat2d_uniform(3, 6), S.heat3d_bumps(3, 4)])
def test_saddle_point_brute_force_nonuniform(prob):
    """Dense solve of the saddle-point system (§2, eq. 2.7) with tau_n reproduces the stepping
    solution in its second component, with p = -u."""
    p = _with_steps(prob, seed=31)
    f, u0 = S.source(p), S.initial(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, taus=p.taus)
    F = T.rhs(f, u0)
    sol = np.linalg.solve(st.dense_saddle(T), np.concatenate([-F.ravel(), -F.ravel()]))
    pp, uu = sol[: F.size].reshape(F.shape), sol[F.size:].reshape(F.shape)
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0, taus=p.taus)
    scale = np.abs(ref).max()
    assert np.abs(uu - ref).max() <= 1e-12 * scale
    assert np.abs(pp + ref).max() <= 1e-12 * scale


def test_equal_steps_reduce_to_the_uniform_oracle():
    p = S.heat2d_uniform(7, 8)
    f = S.source(p)
    a = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f)
    b = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, taus=np.full(p.N, p.T / p.N))
    assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


def test_reference_operator_is_the_time_mean():
    """Abar is the operator of (1/T) int_0^T a dt (eq. 2.2, an average): A itself for a coefficient
    constant in time; for sin(pi t) over (0, 1/2) the operator at the time t* with
    sin(pi t*) = 2/pi; for the workloads' periodic coefficients the a0-only operator, which is also
    the mean of the A_n over uniform steps."""
    p = _with_steps(S.heat2d_uniform(7, 16), seed=4)
    c = dataclasses.replace(p.coeff, ft=S.TRIG_ONE, mt=0.0)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, c, taus=p.taus)
    assert abs(sum(p.taus) - p.T) < 1e-14
    assert abs((T.Abar - T.A[0]).toarray()).max() < 1e-12 * abs(T.A[0].toarray()).max()
    s = dataclasses.replace(p.coeff, ft=S.TRIG_SIN, mt=1.0)
    t_star = math.asin(2.0 / math.pi) / math.pi
    ref = st.assemble_A(2, p.n, s, t_star).toarray()
    assert abs(st.reference_operator(2, p.n, s, 0.5).toarray() - ref).max() < 1e-13 * abs(ref).max()
    for q in (S.heat2d_uniform(7, 16), S.heat3d_bumps(3, 8)):
        a0_only = st.assemble_A(q.dim, q.n, dataclasses.replace(q.coeff, c=0.0), 0.0).toarray()
        Tq = st.SpaceTime(q.dim, q.n, q.N, q.T, q.coeff)
        assert abs(Tq.Abar.toarray() - a0_only).max() < 1e-13 * abs(a0_only).max()
        assert abs((sum(Tq.A) / q.N).toarray() - a0_only).max() < 1e-13 * abs(a0_only).max()


@pytest.mark.parametrize("use_mg", [False, True])
def test_uzawa_nonuniform_reaches_the_stepping_solution(use_mg):
    """Inexact Uzawa (§3, eq. 3.1) with the reference pair (T/N, Abar) of eq. 2.2 converges to
    the implicit-Euler solution on random steps (alpha of eq. 2.2 includes max tau_n/tau)."""
    p = _with_steps(S.heat2d_uniform(15, 32), seed=8)
    f = S.source(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, taus=p.taus)
    F = T.rhs(f, None)
    if use_mg:
        Asolve, Hsolve = mg.st_vcycles(T)
    else:
        Asolve, Hsolve = T.exact_A_solver(), T.exact_H_solver()
    u, _, hist = T.uzawa(F, 0.4, 400, Asolve, Hsolve, tol=1e-11)
    assert hist[-1] <= 1e-11
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, taus=p.taus)
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("dim,n", [(1, 31), (2, 15), (3, 7)])
def test_vcycle_is_homogeneous_of_degree_minus_one(dim, n):
    """The V-cycle reading (weighted Jacobi, full weighting, rediscretised coarse operators, exact
    coarsest solve) of c L is (1/c) times that of L: the property that lets the library run the
    V-cycles of tau A_n for every step and scale the A~ input by rho_n = tau / tau_n (§3, the
    block-diagonal A~ of diag(tau_n A_n))."""
    p = _with_steps(S.heat2d_uniform(n, 6) if dim == 2 else (S.heat1d_mms(n, 6) if dim == 1 else S.heat3d_bumps(n, 6)),
                    seed=12)
    tau = p.T / p.N
    times = np.cumsum(p.taus)

    def build(scales):
        return lambda m: [scales[i] * st.assemble_A(dim, [m] * dim, p.coeff, times[i]) for i in range(p.N)]
    Vn = mg.VCycle(dim, n, build(p.taus))
    Vr = mg.VCycle(dim, n, build(np.full(p.N, tau)))
    r = np.random.default_rng(2).standard_normal((p.N, n ** dim))
    a = Vn.apply(r)
    b = (tau / p.taus)[:, None] * Vr.apply(r)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    # and the scaling is not trivially satisfied: tau_n differ from tau by up to ~25 %
    assert np.abs(p.taus / tau - 1).max() > 0.1
