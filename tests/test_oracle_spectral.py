"""Pins of the oracle's temporal basis, preconditioner and Uzawa iteration (no GPU):
printed values (Table 1), exact identities (Lemma 7.3), a library special case
(scipy.fft DST-II/III), and the paper's bounds (Theorems 3.1 and 4.1, Corollary 6.3)."""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.linalg as sla

import oracle
import synthetic as S
from oracle import mg
from oracle import spacetime as st
from tests.conftest import read_golden

TABLE1 = [(int(r[0]), int(r[1]), float(r[2]), float(r[3]), float(r[4])) for r in read_golden("table1.txt")]


@pytest.mark.parametrize("row", [r for r in TABLE1 if r[0] * r[1] <= 64 * 32 or (r[0] == 128 and r[1] <= 16)])
def test_table1_printed_eigenvalues(row):
    """lambda_min / lambda_max of H^-1 S as printed in Table 1 (§8.1), to the 4 printed digits."""
    hinv, N, lmin, lmax, kappa = row
    a, b = st.table1_eigs(1.0 / hinv, N)
    assert abs(a - lmin) <= 6e-5
    assert abs(b - lmax) <= 6e-5
    assert abs(b / a - kappa) <= 2e-4


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 17, 64, 97])
def test_dst_discrete_orthogonality(N):
    """Lemma 7.3: sum_n w_n phi_k^n phi_j^n = N/2 delta_kj and
    sum_n (phi_k^n - phi_k^{n-1})(phi_j^n - phi_j^{n-1}) = N/2 mu_k^2 delta_kj."""
    V = st.phi_inv(N)  # V[n-1, k-1] = phi_k^n
    w = np.ones(N)
    w[-1] = 0.5
    G = V.T @ (w[:, None] * V)
    assert np.allclose(G, 0.5 * N * np.eye(N), atol=1e-12 * N)
    D = V - np.vstack([np.zeros((1, N)), V[:-1]])
    G2 = D.T @ D
    assert np.allclose(G2, 0.5 * N * np.diag(st.mu(N) ** 2), atol=1e-12 * N)
    assert np.allclose(st.phi(N) @ V, np.eye(N), atol=1e-12)


@pytest.mark.parametrize("N", [1, 4, 7, 64, 100])
def test_dst_matches_library_types(N):
    """Phi^-1 is scipy's (unnormalised) DST-II / 2; Phi^-T is DST-III / 2 of r with r_N
    doubled; Phi is DST-III / N."""
    rng = np.random.default_rng(N)
    y = rng.standard_normal(N)
    assert np.allclose(st.dst_inverse(y[:, None])[:, 0], scipy.fft.dst(y, type=2) / 2, atol=1e-12)
    r = rng.standard_normal(N)
    r2 = r.copy()
    r2[-1] *= 2
    assert np.allclose(st.dst_forward(r[:, None])[:, 0], scipy.fft.dst(r2, type=3) / 2, atol=1e-12)
    assert np.allclose(st.phi(N) @ r, scipy.fft.dst(r, type=3) / N, atol=1e-12)


def _alpha(A_list, Aref):
    lo, hi = np.inf, 0.0
    for A in A_list:
        lam = sla.eigh(A, Aref, eigvals_only=True)
        lo, hi = min(lo, lam[0]), max(hi, lam[-1])
    return max(hi, 1.0 / lo)


@pytest.mark.parametrize("prob", [S.heat1d_mms(15, 16), S.heat2d_uniform(7, 8)])
def test_spectral_equivalence_bounds_variable_coefficient(prob):
    """Theorem 4.1: 1/(2 alpha) H <= S <= 3 alpha H, alpha from eq. 2.2 with Aref = Abar."""
    p = prob
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    A_list = [a.toarray() for a in T.A]
    Aref = T.Abar.toarray()
    S_, H = st.dense_S_H(np.eye(T.ns), A_list, [T.tau] * p.N, Aref, T.tau)
    lam = sla.eigh(S_, H, eigvals_only=True)
    alpha = _alpha(A_list, Aref)
    assert lam[0] >= 1.0 / (2 * alpha) - 1e-10
    assert lam[-1] <= 3 * alpha + 1e-10


def test_schur_complement_symmetric_positive_definite_and_max_norm_bound():
    """Theorem 6.2 (S symmetric positive definite) and Corollary 6.3
    (max_n ||u_n||_M <= ||u||_S) for a variable-coefficient FD problem."""
    p = S.heat2d_uniform(7, 6)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    N, m = p.N, T.ns
    Kb = np.kron(st.K_matrix(N), np.eye(m))
    Ab = sla.block_diag(*[T.tau * a.toarray() for a in T.A])
    Sm = Kb.T @ np.linalg.solve(Ab, Kb) + Kb + Kb.T + Ab
    assert np.abs(Sm - Sm.T).max() <= 1e-10 * np.abs(Sm).max()
    assert np.linalg.eigvalsh(0.5 * (Sm + Sm.T)).min() > 0
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.standard_normal(N * m)
        snorm = math.sqrt(u @ Sm @ u)
        assert np.linalg.norm(u.reshape(N, m), axis=1).max() <= snorm * (1 + 1e-12)


def test_uzawa_exact_solvers_reaches_oracle_and_p_is_minus_u():
    p = S.heat2d_uniform(7, 16)
    f = S.source(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    F = T.rhs(f, None)
    u, pp, hist = T.uzawa(F, 0.55, 300, T.exact_A_solver(), T.exact_H_solver(), tol=1e-12)
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(pp + ref) <= 1e-10 * np.linalg.norm(ref)


def _rho_uzawa(rho_a, omega, lmin, lmax):
    """sigma_-, sigma_+ and rho_U of Theorem 3.1 (eq. 3.5)."""
    sm = 0.5 * ((1 - rho_a) * (1 - omega * lmin) + math.sqrt(4 * rho_a + (1 - rho_a) ** 2 * (1 - omega * lmin) ** 2))
    c = (1 + rho_a) * (1 + omega * lmax) - 2
    sp_ = 0.5 * (c + math.sqrt(4 * rho_a + c * c))
    return max(sm, sp_)


@pytest.mark.parametrize("use_mg", [False, True])
def test_uzawa_contraction_bound(use_mg):
    """Theorem 3.1: ||e_{j+1}||_D <= rho_U ||e_j||_D with
    ||(q, v)||_D^2 = omega rho_A ||q||^2_{A~} + ||v||^2_{H~} (eq. 3.4, 3.6)."""
    p = S.heat1d_mms(7, 8)
    f, u0 = S.source(p), S.initial(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    F = T.rhs(f, u0)
    N, m = p.N, T.ns
    if use_mg:
        Asolve, Hsolve = mg.st_vcycles(T, h_cycles=1)
    else:
        Asolve, Hsolve = T.exact_A_solver(), T.exact_H_solver()
    # dense A~^-1 (block diagonal) and H~^-1 from the solvers' actions on unit vectors
    E = np.eye(N * m).reshape(N * m, N, m)
    Ainv_t = np.stack([Asolve(E[i]).ravel() for i in range(N * m)], axis=1)
    Hinv = np.stack([T.apply_Hinv(E[i], Hsolve).ravel() for i in range(N * m)], axis=1)
    Ainv_t, Hinv = 0.5 * (Ainv_t + Ainv_t.T), 0.5 * (Hinv + Hinv.T)
    Atil, Htil = np.linalg.inv(Ainv_t), np.linalg.inv(Hinv)
    Ab = sla.block_diag(*[T.tau * a.toarray() for a in T.A])
    Kb = np.kron(st.K_matrix(N), np.eye(m))
    Sm = Kb.T @ np.linalg.solve(Ab, Kb) + Kb + Kb.T + Ab
    lam = sla.eigh(0.5 * (Sm + Sm.T), Htil, eigvals_only=True)
    rho_a = np.abs(1 - np.linalg.eigvals(Ainv_t @ Ab)).max() if use_mg else 0.0
    assert rho_a < 1
    omega = 0.9 * 2 * (1 - rho_a) / ((1 + rho_a) * lam[-1])
    rho_u = _rho_uzawa(rho_a, omega, lam[0], lam[-1])
    assert rho_u < 1
    uex = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0).ravel()
    pex = -uex

    def dnorm(q, v):
        return math.sqrt(omega * rho_a * (q @ Atil @ q) + v @ Htil @ v)

    u = np.zeros(N * m)
    pv = np.zeros(N * m)
    prev = dnorm(pex - pv, uex - u)
    for _ in range(12):
        rp = Kb @ u - Ab @ pv - F.ravel()
        pv = pv + Ainv_t @ rp
        ru = F.ravel() - Kb.T @ pv - (Kb + Kb.T + Ab) @ u
        u = u + omega * Hinv @ ru
        cur = dnorm(pex - pv, uex - u)
        assert cur <= rho_u * prev * (1 + 1e-8) + 1e-13
        prev = cur


@pytest.mark.parametrize("prob", [S.heat2d_uniform(15, 4), S.heat3d_bumps(7, 3), S.heat3d_bumps(15, 2)],
                         ids=lambda p: p.name)
def test_sine_H_solver_equals_sparse_direct_solves(prob):
    """The sine-transform H_k solver that the large 3-D GPU tests use agrees with the sparse direct
    H_k solves of the oracle (§4, eq. 4.4), and so does the whole H~^-1."""
    from tests.conftest import sine_H_solver
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff)
    direct, sine = T.exact_H_solver(), sine_H_solver(T)
    r = np.random.default_rng(11).standard_normal((prob.N, prob.ns))
    for k in range(prob.N):
        a, b = sine(k, r[k]), direct(k, r[k])
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    a, b = T.apply_Hinv(r, sine), T.apply_Hinv(r, direct)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
