"""Pins of the oracle's multigrid V-cycle reading and of the seeded input generator (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as S
from oracle import mg
from oracle import spacetime as st
from tests.conftest import read_golden


def _dense_V(V, ns):
    E = np.eye(ns)
    return np.stack([V.apply_one(0, E[i]) for i in range(ns)], axis=1)


@pytest.mark.parametrize("dim,n", [(1, 31), (2, 15), (3, 7)])
def test_vcycle_symmetric_positive_definite_and_convergent(dim, n):
    """A symmetric V-cycle is a symmetric, positive definite approximate inverse with
    contraction rho_A = max |1 - lambda(V L)| < 1 (§3, eq. 3.3)."""
    coeff = S.heat3d_bumps().coeff if dim == 3 else S.heat2d_uniform().coeff
    L0 = 0.01 * st.assemble_A(dim, [n] * dim, coeff, 0.3)
    V = mg.VCycle(dim, n, lambda m: [0.01 * st.assemble_A(dim, [m] * dim, coeff, 0.3)])
    Vd = _dense_V(V, n ** dim)
    assert np.abs(Vd - Vd.T).max() <= 1e-12 * np.abs(Vd).max()
    assert np.linalg.eigvalsh(0.5 * (Vd + Vd.T)).min() > 0
    rho = np.abs(1 - np.linalg.eigvals(Vd @ L0.toarray())).max()
    assert rho < 0.5


def test_vcycle_iteration_converges_to_direct_solve():
    dim, n = 2, 31
    coeff = S.heat2d_uniform().coeff
    L = 0.002 * st.assemble_A(dim, [n, n], coeff, 0.1) + 0.7 * sp.identity(n * n)
    V = mg.VCycle(dim, n, lambda m: [0.002 * st.assemble_A(dim, [m, m], coeff, 0.1) + 0.7 * sp.identity(m * m)])
    b = np.random.default_rng(0).standard_normal(n * n)
    x = np.zeros_like(b)
    for _ in range(30):
        x = x + V.apply_one(0, b - L @ x)
    xs = sp.linalg.spsolve(L.tocsc(), b)
    assert np.abs(x - xs).max() <= 1e-11 * np.abs(xs).max()


def test_rediscretised_coarse_operator_is_galerkin_in_1d():
    """For the constant-coefficient 1-D operator, R L_h P with R = P^T/2 equals the
    rediscretised L_2h: pins the prolongation weights and the restriction scaling."""
    n = 15
    coeff = S.Coeff(1.7, 0.0)
    Lf = st.assemble_A(1, [n], coeff, 0.0).toarray()
    Lc = st.assemble_A(1, [7], coeff, 0.0).toarray()
    P = mg.prolongation(1, 7).toarray()
    assert np.abs(P.T @ Lf @ P / 2 - Lc).max() <= 1e-12 * np.abs(Lc).max()


def test_prolongation_reproduces_multilinear_functions():
    """d-linear interpolation (zero Dirichlet data) is exact for products of coarse-grid
    tent functions, which are d-linear on every coarse cell and vanish on the boundary."""
    for dim in (1, 2, 3):
        nc = 3
        P = mg.prolongation(dim, nc)
        xc = S.grid_axes(dim, [nc] * dim)
        xf = S.grid_axes(dim, [2 * nc + 1] * dim)

        def field(axes):
            grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
            out = np.ones_like(grids[0])
            for d, g in enumerate(grids):
                out = out * np.minimum(g, 1 - g) * (1 - 0.3 * d)
            return out.ravel()
        assert np.abs(P @ field(xc) - field(xf)).max() < 1e-14


def test_splitmix64_reference_outputs():
    for seed, idx, out in read_golden("splitmix64.txt"):
        assert int(S.splitmix64(int(seed), int(idx))) == int(out)


def test_uniform_inputs_range_and_moments():
    v = S.uniform_pm1(1, 1 << 20)
    assert v.min() >= -1.0 and v.max() < 1.0
    assert abs(v.mean()) < 5e-3 and abs(v.var() - 1.0 / 3.0) < 5e-3
