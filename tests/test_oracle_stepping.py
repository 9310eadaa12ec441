"""Pins of the oracle's time stepping and time-global operators against closed forms,
convergence orders and brute-force dense solves (no GPU)."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import spacetime as st


@pytest.mark.parametrize("dim,n,mode,a0", [(1, 31, (3,), 0.7), (2, 15, (2, 5), 1.3), (3, 7, (1, 2, 3), 2.0)])
def test_eigenmode_decay_closed_form(dim, n, mode, a0):
    """Constant a: u0 = prod sin(m_d pi x_d) is an eigenvector of A with
    lambda_h = sum_d 4 a0 h^-2 sin^2(m_d pi h / 2), so u_n = (1 + tau lambda_h)^-n u0 (§2, eq. 2.1)."""
    p = S.eigenmode(dim, n, 12, 0.3, a0, mode)
    f, u0 = S.source(p), S.initial(p)
    u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0)
    h = 1.0 / (n + 1)
    tau = p.T / p.N
    lam = sum(4 * a0 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2 for m in mode)
    exact = np.stack([(1 + tau * lam) ** (-k) * u0 for k in range(1, p.N + 1)])
    assert np.abs(u - exact).max() < 1e-13


def test_eigenmode_cg_matches_closed_form():
    p = S.eigenmode(3, 7, 6, 0.3, 1.1, (1, 1, 2))
    f, u0 = S.source(p), S.initial(p)
    u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0, method="cg", cg_tol=1e-15)
    h = 1.0 / 8
    tau = p.T / p.N
    lam = sum(4 * 1.1 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2 for m in (1, 1, 2))
    exact = np.stack([(1 + tau * lam) ** (-k) * u0 for k in range(1, p.N + 1)])
    assert np.abs(u - exact).max() < 1e-12


def test_mms_first_order_in_time_second_in_space():
    """The manufactured 1-D problem: error O(tau + h^2); halving h and quartering tau
    divides the max error by ~4."""
    errs = []
    for n, N in [(63, 64), (127, 256)]:
        p = S.heat1d_mms(n, N)
        u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), S.initial(p))
        errs.append(np.abs(u - S.mms1_exact(n, N, p.T)).max())
    assert 1e-4 < errs[0] < 1e-3
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_cg_agrees_with_cholesky_variable_coefficient():
    p = S.heat2d_uniform(15, 6)
    f = S.source(p)
    a = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f)
    b = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, method="cg", cg_tol=1e-15)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    p3 = S.heat3d_bumps(7, 5)
    f3 = S.source(p3)
    a3 = oracle.implicit_euler(p3.dim, p3.n, p3.N, p3.T, p3.coeff, f3)
    b3 = oracle.implicit_euler(p3.dim, p3.n, p3.N, p3.T, p3.coeff, f3, method="cg", cg_tol=1e-15)
    assert np.abs(a3 - b3).max() <= 1e-12 * np.abs(a3).max()


@pytest.mark.parametrize("prob", [S.heat1d_mms(7, 8), S.heat2d_uniform(3, 6), S.heat3d_bumps(3, 4)])
def test_saddle_point_brute_force(prob):
    """Dense solve of the saddle-point system (§2, eq. 2.7) reproduces the
    time-stepping solution in its second component, with p = -u."""
    p = prob
    f, u0 = S.source(p), S.initial(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    F = T.rhs(f, u0)
    Asad = st.dense_saddle(T)
    sol = np.linalg.solve(Asad, np.concatenate([-F.ravel(), -F.ravel()]))
    pp, uu = sol[: F.size].reshape(F.shape), sol[F.size:].reshape(F.shape)
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0)
    scale = np.abs(ref).max()
    assert np.abs(uu - ref).max() <= 1e-12 * scale
    assert np.abs(pp + ref).max() <= 1e-12 * scale


def test_apply_B_matches_assembled_and_stepping():
    """C apply_B agrees with the SciPy-assembled B, and B u = F for the stepped u."""
    p = S.heat2d_uniform(7, 5)
    f = S.source(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    rng = np.random.default_rng(0)
    v = rng.standard_normal((p.N, p.ns))
    assert np.abs(oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, v) - T.B(v)).max() < 1e-12
    u = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f)
    F = T.rhs(f, None)
    assert np.abs(oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, u) - F).max() < 1e-13


def test_assembled_A_is_symmetric_positive_definite():
    p = S.heat3d_bumps(3, 4)
    A = st.assemble_A(3, p.n, p.coeff, 0.37).toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
