"""Plain NumPy/SciPy statement of the paper's time-global objects (test infrastructure only).

Everything here is written straight from the paper's definitions, at sizes
where dense or sparse-direct linear algebra finishes in seconds:

* the finite-difference spatial operators A_n (conservative, coefficient at face
  midpoints, Dirichlet) at t_n = tau_1 + ... + tau_n, the reference pair
  tau = T/N and Abar = the operator of the coefficient's time mean over (0, T)
  (one of the averages §2 allows after eq. 2.2),
* the mass matrix M of eq. 2.1: the identity (finite differences) or the P1 finite-element mass
  matrix of the uniform mesh divided by h^d (1-D and 2-D, the 2-D mesh cutting every square along
  its lower-left to upper-right diagonal); the P1 stiffness matrix with the coefficient at the edge
  midpoints is h^d times the finite-difference operator, so the finite-element system divided by
  h^d uses the same A_n,
* the time-global matrices K, B = K (x) M + diag(tau_n A_n) (§2, eq. 2.3-2.4),
  the Schur complement S (eq. 2.5) and the saddle-point matrix (eq. 2.7),
* the temporal change of basis Phi (type-III DST, §4 eq. 4.2), its inverse
  (type-II DST, eq. 4.3) and mu_k (eq. 4.5),
* the preconditioner H = Phi^T Hhat Phi, Hhat = N/(2 tau) diag(H_k A^-1 H_k)
  (eq. 4.4), and its inverse applied as Phi^-1 Hhat^-1 Phi^-T,
* the inexact Uzawa iteration (§3, eq. 3.1) with caller-supplied spatial
  solvers (exact sparse LU, or the multigrid V-cycle of ``oracle.mg``).

No blocking, fusion or reordering beyond what those definitions state.
"""
from __future__ import annotations

import math
import types
from typing import Callable, List, Optional, Sequence

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _trig(kind: int, arg):
    if kind == 1:
        return np.sin(arg)
    if kind == 2:
        return np.cos(arg)
    return np.ones_like(np.asarray(arg, dtype=np.float64))


def coefficient(coeff, coords: Sequence[np.ndarray], t: float) -> np.ndarray:
    """a(x,t) = a0 + c * prod_d g_d(pi m_d x_d) * g_t(pi m_t t) at the given coordinates."""
    g = coeff.c * _trig(coeff.ft, math.pi * coeff.mt * t) * np.ones_like(coords[0])
    for d, x in enumerate(coords):
        g = g * _trig(coeff.fx[d], math.pi * coeff.mx[d] * x)
    return coeff.a0 + g


def grid_index(dim: int, n: Sequence[int]):
    """Per-point 0-based axis indices, x fastest."""
    ns = int(np.prod(n[:dim]))
    idx = np.arange(ns)
    out = []
    for d in range(dim):
        out.append(idx % n[d])
        idx = idx // n[d]
    return out


def assemble_A(dim: int, n: Sequence[int], coeff, t: float) -> sp.csr_matrix:
    """FD operator (A v)_i = sum_d h^-2 [a_-(v_i - v_{i-e_d}) + a_+(v_i - v_{i+e_d})]."""
    n = list(n)[:dim]
    ns = int(np.prod(n))
    ix = grid_index(dim, n)
    h = [1.0 / (m + 1) for m in n]
    strides = [int(np.prod(n[:d])) for d in range(dim)]
    diag = np.zeros(ns)
    rows, cols, vals = [], [], []
    for d in range(dim):
        # face between node j and j+1 (nodes 0 and n+1 on the boundary) is at (j + 1/2) h
        def face_coef(shift):
            coords = [(ix[e] + 1) * h[e] for e in range(dim)]
            coords[d] = (ix[d] + shift) * h[d]
            return coefficient(coeff, coords, t)
        am = face_coef(0.5)
        ap = face_coef(1.5)
        diag += (am + ap) / h[d] ** 2
        has_up = ix[d] < n[d] - 1
        i = np.nonzero(has_up)[0]
        j = i + strides[d]
        v = -ap[i] / h[d] ** 2
        rows += [i, j]
        cols += [j, i]
        vals += [v, v]
    rows.append(np.arange(ns))
    cols.append(np.arange(ns))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(ns, ns))


def assemble_M(dim: int, n: Sequence[int], mass: str = "identity") -> sp.csr_matrix:
    """The mass matrix of eq. 2.1 over h^d: the identity, or for "p1" the P1 mass matrix of the
    uniform mesh (1-D: h [1/6, 2/3, 1/6]; 2-D, squares cut along the lower-left to upper-right
    diagonal: h^2/2 at the point, h^2/12 at the four axis neighbours and at the upper-right and
    lower-left ones) divided by h^d."""
    n = list(n)[:dim]
    ns = int(np.prod(n))
    if mass == "identity":
        return sp.identity(ns, format="csr")
    if mass != "p1" or dim > 2:
        raise ValueError("mass %r in %d-D" % (mass, dim))
    if dim == 1:
        m = n[0]
        return sp.diags([np.full(m - 1, 1 / 6), np.full(m, 2 / 3), np.full(m - 1, 1 / 6)], [-1, 0, 1],
                        format="csr")
    x, y = grid_index(dim, n)
    rows, cols, vals = [np.arange(ns)], [np.arange(ns)], [np.full(ns, 0.5)]
    for dx, dy in ((1, 0), (0, 1), (1, 1)):  # each coupling once, then mirrored
        i = np.nonzero((x + dx < n[0]) & (y + dy < n[1]))[0]
        j = i + dx + dy * n[0]
        rows += [i, j]
        cols += [j, i]
        vals += [np.full(i.size, 1 / 12), np.full(i.size, 1 / 12)]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(ns, ns))


def K_matrix(N: int) -> np.ndarray:
    """Lower bidiagonal [1; -1 1] of §2, eq. 2.4."""
    return np.eye(N) - np.eye(N, k=-1)


def phi(N: int) -> np.ndarray:
    """Phi[k-1, n-1] = (2/N) (1 + delta_{nN})^-1 sin((2k-1) n pi / (2N))  (§4, eq. 4.2)."""
    k = np.arange(1, N + 1)[:, None]
    n = np.arange(1, N + 1)[None, :]
    w = np.where(n == N, 0.5, 1.0)
    return (2.0 / N) * w * np.sin((2 * k - 1) * n * math.pi / (2 * N))


def phi_inv(N: int) -> np.ndarray:
    """Phi^-1[n-1, k-1] = sin((2k-1) n pi / (2N))  (§4, eq. 4.3)."""
    n = np.arange(1, N + 1)[:, None]
    k = np.arange(1, N + 1)[None, :]
    return np.sin((2 * k - 1) * n * math.pi / (2 * N))


def mu(N: int) -> np.ndarray:
    """mu_k = 2 sin((2k-1) pi / (4N)), k = 1..N  (§4, eq. 4.5)."""
    k = np.arange(1, N + 1)
    return 2.0 * np.sin((2 * k - 1) * math.pi / (4 * N))


def dst_forward(r: np.ndarray) -> np.ndarray:
    """rhat = Phi^-T r, i.e. rhat_k = sum_n r_n sin((2k-1) n pi/(2N)); r is [N][...]."""
    N = r.shape[0]
    return phi_inv(N).T @ r.reshape(N, -1)


def dst_inverse(y: np.ndarray) -> np.ndarray:
    """u = Phi^-1 y, i.e. u_n = sum_k y_k sin((2k-1) n pi/(2N)); y is [N][...]."""
    N = y.shape[0]
    return phi_inv(N) @ y.reshape(N, -1)


def step_times(N: int, T: float, taus=None):
    """(tau_n, t_n) for n = 1..N: uniform tau = T/N, t_n = n tau, or the given step lengths with
    t_n = tau_1 + ... + tau_n (§2, before eq. 2.1)."""
    if taus is None:
        tau = T / N
        return np.full(N, tau), np.array([(i + 1) * tau for i in range(N)])
    taus = np.asarray(taus, dtype=np.float64).reshape(-1)
    assert taus.size == N and np.all(taus > 0)
    return taus.copy(), np.cumsum(taus)


def time_mean_factor(coeff, T: float, pieces: int = 64) -> float:
    """(1/T) int_0^T g_t(pi m_t t) dt: composite 32-point Gauss-Legendre quadrature."""
    x, w = np.polynomial.legendre.leggauss(32)
    edges = np.linspace(0.0, T, pieces + 1)
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        t = 0.5 * (b - a) * x + 0.5 * (a + b)
        total += 0.5 * (b - a) * float(np.dot(w, _trig(coeff.ft, math.pi * coeff.mt * t)))
    return total / T


def reference_operator(dim: int, n: Sequence[int], coeff, T: float) -> sp.csr_matrix:
    """Abar (eq. 2.2, "an average"): the FD operator of the time mean of the coefficient over (0, T),
    a0 + c gbar prod_d g_d(pi m_d x_d) with gbar = (1/T) int_0^T g_t; it does not depend on the
    time grid (for uniform steps and a coefficient periodic over (0, T) it is the mean of the A_n)."""
    gbar = time_mean_factor(coeff, T)
    mean = types.SimpleNamespace(a0=coeff.a0, c=coeff.c * gbar, fx=coeff.fx, mx=coeff.mx, ft=0, mt=0.0)
    return assemble_A(dim, n, mean, 0.0)


class SpaceTime:
    """The time-global problem: grid, N steps tau_n (uniform T/N unless ``taus`` is given), the
    mass matrix M (``mass``: "identity" for finite differences, "p1" for P1 finite elements, see
    assemble_M); the reference step of the preconditioner is tau = T/N."""

    def __init__(self, dim: int, n: Sequence[int], N: int, T: float, coeff, taus=None, mass="identity"):
        self.dim, self.n, self.N, self.T, self.coeff = dim, list(n)[:dim], N, float(T), coeff
        self.mass = mass
        self.M = assemble_M(dim, self.n, mass)
        self.tau = self.T / N
        self.uniform = taus is None
        self.taus, self.times = step_times(N, self.T, taus)
        self.ns = int(np.prod(self.n))
        self.A = [assemble_A(dim, self.n, coeff, self.times[i]) for i in range(N)]
        self.Abar = reference_operator(dim, self.n, coeff, self.T)

    # -- time-global operators (vectors are [N][ns]) --
    def K(self, u):
        """(K (x) M) u: M (u_n - u_{n-1}), u_0 := 0."""
        out = u.copy()
        out[1:] -= u[:-1]
        return (self.M @ out.T).T

    def Kt(self, p):
        """(K^T (x) M) p: M (p_n - p_{n+1}), p_{N+1} := 0."""
        out = p.copy()
        out[:-1] -= p[1:]
        return (self.M @ out.T).T

    def Ablk(self, v):
        return np.stack([self.taus[i] * (self.A[i] @ v[i]) for i in range(self.N)])

    def B(self, u):
        return self.K(u) + self.Ablk(u)

    def rhs(self, f: np.ndarray, u0: Optional[np.ndarray]) -> np.ndarray:
        """F = [tau_1 f_1 + M u_I, tau_2 f_2, ..., tau_N f_N]  (§2, after eq. 2.4), the load f_n
        being M times the nodal values given (the identity for finite differences)."""
        F = self.taus[:, None] * np.asarray(f, dtype=np.float64).reshape(self.N, self.ns)
        if u0 is not None:
            F[0] += u0
        return np.ascontiguousarray((self.M @ F.T).T)

    def residual(self, F, u):
        return np.linalg.norm(F - self.B(u)) / np.linalg.norm(F)

    # -- exact spatial solvers --
    def exact_A_solver(self) -> Callable:
        lus = [spla.splu((self.taus[i] * self.A[i]).tocsc()) for i in range(self.N)]

        def solve(r):
            return np.stack([lus[i].solve(r[i]) for i in range(self.N)])
        return solve

    def exact_H_solver(self) -> Callable:
        m = mu(self.N)
        lus = [spla.splu((m[k] * self.M + self.tau * self.Abar).tocsc()) for k in range(self.N)]

        def solve(k, r):
            return lus[k].solve(r)
        return solve

    def apply_Hinv(self, r: np.ndarray, Hsolve: Callable) -> np.ndarray:
        """Phi^-1 Hhat^-1 Phi^-T r with Hhat_k^-1 = (2 tau / N) H_k^-1 Abar H_k^-1 (§4, eq. 4.4/4.6)."""
        rhat = dst_forward(r)
        y = np.empty_like(rhat)
        for k in range(self.N):
            z = Hsolve(k, rhat[k])
            y[k] = (2.0 * self.tau / self.N) * Hsolve(k, self.Abar @ z)
        return dst_inverse(y)

    def uzawa(self, F: np.ndarray, omega: float, max_it: int, Asolve: Callable,
              Hsolve: Callable, tol: float = 0.0):
        """Inexact Uzawa (§3, eq. 3.1) from u_0 = p_0 = 0.

        Returns (u, p, hist) where hist[j] = ||F - B u_j|| / ||F|| and the loop stops at the
        first j with hist[j] <= tol (returning u_j) or after max_it updates.
        """
        u = np.zeros((self.N, self.ns))
        p = np.zeros_like(u)
        hist = []
        for j in range(max_it + 1):
            hist.append(self.residual(F, u))
            if hist[-1] <= tol or j == max_it:
                break
            rp = self.K(u) - self.Ablk(p) - F
            p = p + Asolve(rp)
            ru = F - self.Kt(p) - (self.K(u) + self.Kt(u) + self.Ablk(u))
            u = u + omega * self.apply_Hinv(ru, Hsolve)
        return u, p, np.array(hist)


# ---- dense objects for spectral checks (small sizes only) -------------------------

def dense_S_H(M: np.ndarray, A_list: List[np.ndarray], tau_list: Sequence[float], Aref: np.ndarray,
              tau: float):
    """Dense S = K^T A^-1 K + K + K^T + A (eq. 2.5) and H = Phi^T Hhat Phi (eq. 4.4).

    Bold K = K (x) M, bold A = diag(tau_n A_n); H_k = mu_k M + tau Aref.
    """
    N = len(A_list)
    m = M.shape[0]
    Kb = np.kron(K_matrix(N), M)
    Ab = sla.block_diag(*[tau_list[i] * A_list[i] for i in range(N)])
    S = Kb.T @ np.linalg.solve(Ab, Kb) + Kb + Kb.T + Ab
    mus = mu(N)
    Aref_inv = np.linalg.inv(Aref)
    blocks = []
    for k in range(N):
        Hk = mus[k] * M + tau * Aref
        blocks.append((N / (2.0 * tau)) * Hk @ Aref_inv @ Hk)
    Hhat = sla.block_diag(*blocks)
    Phib = np.kron(phi(N), np.eye(m))
    H = Phib.T @ Hhat @ Phib
    return 0.5 * (S + S.T), 0.5 * (H + H.T)


def fem1d_matrices(h: float):
    """P1 FEM mass and stiffness on (0,1), uniform mesh h, interior nodes (§8.1 setting)."""
    m = int(round(1.0 / h)) - 1
    M = (h / 6.0) * (4 * np.eye(m) + np.eye(m, k=1) + np.eye(m, k=-1))
    A = (1.0 / h) * (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1))
    return M, A


def table1_eigs(h: float, N: int, T: float = 1.0):
    """Extremal eigenvalues of H^-1 S for the 1-D P1 heat problem of §8.1 (Table 1)."""
    M, A = fem1d_matrices(h)
    tau = T / N
    S, H = dense_S_H(M, [A] * N, [tau] * N, A, tau)
    lam = sla.eigh(S, H, eigvals_only=True)
    return lam[0], lam[-1]


def dense_saddle(st: SpaceTime):
    """The saddle-point matrix [[A, -K], [-K^T, -(K + K^T + A)]] of §2, eq. 2.7 (dense)."""
    N, ns = st.N, st.ns
    Kb = np.kron(K_matrix(N), st.M.toarray())
    Ab = sla.block_diag(*[st.taus[i] * st.A[i].toarray() for i in range(N)])
    top = np.hstack([Ab, -Kb])
    bot = np.hstack([-Kb.T, -(Kb + Kb.T + Ab)])
    return np.vstack([top, bot])
