"""Plain statement of the geometric-multigrid V-cycle used for the spatial solves.

Test infrastructure only.  The paper states only that the spatial solvers are
"one or two MG V-cycles with Jacobi smoothers" (§8.2) and that each must be a
symmetric positive definite, convergent approximation of its operator (§3,
eq. 3.3; §4, eq. 4.7).  The reading implemented here (and by the GPU path) is:

* grids with n_l interior points per axis, n_{l+1} = (n_l - 1)/2, down to one point;
* level operator L_l = sigma M_l + s A_l, where A_l is the finite-difference operator
  of the same coefficient field sampled at level-l face midpoints (rediscretised) and M_l the
  mass matrix of the problem over h^d at level l (the identity, or the P1 stencil);
* prolongation P = d-linear interpolation, restriction R = P^T / 2^d (full weighting);
* V(1,1): one weighted-Jacobi sweep x <- x + w D^-1 (b - L x) before and after the
  coarse-grid correction, w = 2/3, 4/5, 6/7 for d = 1, 2, 3; exact solve on the
  one-point grid; zero initial guess.

With R proportional to P^T and the same symmetric smoother before and after, the
V-cycle is a symmetric linear map of b.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np
import scipy.sparse as sp

JACOBI_WEIGHT = {1: 2.0 / 3.0, 2: 4.0 / 5.0, 3: 6.0 / 7.0}


def level_sizes(n: int) -> List[int]:
    sizes = [n]
    while sizes[-1] > 1:
        if sizes[-1] % 2 == 0:
            raise ValueError("n + 1 must be a power of two, got n = %d" % n)
        sizes.append((sizes[-1] - 1) // 2)
    return sizes


def prolongation_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc coarse to 2 nc + 1 fine interior points."""
    nf = 2 * nc + 1
    rows, cols, vals = [], [], []
    for m in range(nc):
        f = 2 * m + 1
        rows += [f - 1, f, f + 1]
        cols += [m, m, m]
        vals += [0.5, 1.0, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(dim: int, nc: int) -> sp.csr_matrix:
    P1 = prolongation_1d(nc)
    P = P1
    for _ in range(dim - 1):
        P = sp.kron(P1, P, format="csr")  # slower axes to the left: x fastest
    return P


class VCycle:
    """Batched symmetric V(1,1) for B independent slices sharing one grid.

    ``build(level_n) -> list of B sparse matrices`` gives the level operators.
    """

    def __init__(self, dim: int, n: int, build: Callable[[int], Sequence[sp.spmatrix]],
                 weight: float = None):
        self.dim = dim
        self.sizes = level_sizes(n)
        self.w = JACOBI_WEIGHT[dim] if weight is None else weight
        self.L = []
        self.Dinv = []
        for m in self.sizes:
            ops = list(build(m))
            self.L.append(ops)
            self.Dinv.append([1.0 / op.diagonal() for op in ops])
        self.P = [prolongation(dim, self.sizes[l + 1]) for l in range(len(self.sizes) - 1)]
        self.B = len(self.L[0])

    def _cycle(self, l: int, b: int, rhs: np.ndarray) -> np.ndarray:
        L = self.L[l][b]
        if l == len(self.sizes) - 1:
            return rhs / L.diagonal()  # one point: exact
        Dinv = self.Dinv[l][b]
        x = self.w * Dinv * rhs                      # pre-smoothing from x = 0
        r = rhs - L @ x
        rc = (self.P[l].T @ r) / (2 ** self.dim)     # full weighting
        ec = self._cycle(l + 1, b, rc)
        x = x + self.P[l] @ ec                       # coarse-grid correction
        x = x + self.w * Dinv * (rhs - L @ x)        # post-smoothing
        return x

    def apply(self, rhs: np.ndarray) -> np.ndarray:
        """rhs is [B][ns]; returns V(rhs) slice by slice."""
        return np.stack([self._cycle(0, b, rhs[b]) for b in range(self.B)])

    def apply_one(self, b: int, rhs: np.ndarray) -> np.ndarray:
        return self._cycle(0, b, rhs)


def st_vcycles(st, h_cycles: int = 2):
    """V-cycle solvers for the Uzawa preconditioners of a ``SpaceTime`` problem.

    Returns (Asolve, Hsolve): Asolve applies, slice n, one V-cycle for tau_n A_n
    (coefficient at t_n, step length tau_n); Hsolve(k, r) applies ``h_cycles`` steps of the V-cycle iteration
    x <- x + V(r - H_k x) from x = 0 for H_k = mu_k M + tau Abar.
    """
    from .spacetime import assemble_A, assemble_M, mu, reference_operator

    dim, n, N, tau = st.dim, st.n[0], st.N, st.tau

    def build_A(m):
        return [st.taus[i] * assemble_A(dim, [m] * dim, st.coeff, st.times[i]) for i in range(N)]

    mus = mu(N)

    def build_H(m):
        Abar = reference_operator(dim, [m] * dim, st.coeff, st.T)
        M = assemble_M(dim, [m] * dim, getattr(st, "mass", "identity"))
        return [mus[k] * M + tau * Abar for k in range(N)]

    VA = VCycle(dim, n, build_A)
    VH = VCycle(dim, n, build_H)

    def Hsolve(k, r):
        x = VH.apply_one(k, r)
        for _ in range(h_cycles - 1):
            x = x + VH.apply_one(k, r - VH.L[0][k] @ x)
        return x
    return VA.apply, Hsolve
