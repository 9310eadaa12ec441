"""Pins of the oracle's P1 finite-element form (M != I in §2, eq. 2.1): the mass and stiffness
stencils against a brute-force element-by-element assembly, the closed-form decay of a 1-D
eigenmode, the dense saddle-point solve, the order of convergence on a manufactured 2-D solution,
and the Uzawa iteration converging to the stepped solution (no GPU)."""
import math
import types

import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import mg
from oracle import spacetime as st

ONE = types.SimpleNamespace(a0=1.0, c=0.0, fx=[0, 0, 0], mx=[0.0] * 3, ft=0, mt=0.0)


def element_assembly(dim, n):
    """P1 mass and stiffness (a = 1) of the uniform mesh of (0,1)^dim with n interior points per
    axis, summed element by element from the textbook element matrices: on an interval of length h,
    mass (h/6)[2 1; 1 2] and stiffness (1/h)[1 -1; -1 1]; on a triangle of area |T|, mass
    (|T|/12)(1 + delta_ij) and stiffness |T| grad(phi_i).grad(phi_j).  Squares are cut along the
    diagonal from the lower-left to the upper-right corner.  Boundary nodes are dropped."""
    h = 1.0 / (n + 1)
    ns = n ** dim
    M = np.zeros((ns, ns))
    K = np.zeros((ns, ns))

    def idx(*c):  # interior index of a node, or None on the boundary
        if any(v < 1 or v > n for v in c):
            return None
        out, mul = 0, 1
        for v in c:
            out += (v - 1) * mul
            mul *= n
        return out

    if dim == 1:
        Me = (h / 6) * np.array([[2, 1], [1, 2]])
        Ke = (1 / h) * np.array([[1, -1], [-1, 1]])
        for e in range(n + 1):
            nodes = [idx(e), idx(e + 1)]
            for a in range(2):
                for b in range(2):
                    if nodes[a] is not None and nodes[b] is not None:
                        M[nodes[a], nodes[b]] += Me[a, b]
                        K[nodes[a], nodes[b]] += Ke[a, b]
        return M, K
    for i in range(n + 1):
        for j in range(n + 1):
            corners = {"sw": (i, j), "se": (i + 1, j), "ne": (i + 1, j + 1), "nw": (i, j + 1)}
            for tri in (("sw", "se", "ne"), ("sw", "ne", "nw")):
                pts = np.array([corners[c] for c in tri], dtype=float) * h
                e1, e2 = pts[1] - pts[0], pts[2] - pts[0]
                area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
                # gradients of the barycentric functions: solve [x y 1] c = e_k
                V = np.hstack([pts, np.ones((3, 1))])
                G = np.linalg.inv(V)[:2, :].T  # row k = grad(phi_k)
                nodes = [idx(*corners[c]) for c in tri]
                for a in range(3):
                    for b in range(3):
                        if nodes[a] is None or nodes[b] is None:
                            continue
                        M[nodes[a], nodes[b]] += area / 12 * (2 if a == b else 1)
                        K[nodes[a], nodes[b]] += area * G[a] @ G[b]
    return M, K


@pytest.mark.parametrize("dim,n", [(1, 3), (1, 7), (2, 3), (2, 7)])
def test_p1_stencils_equal_element_assembly(dim, n):
    """h^d times the oracle's mass over h^d and h^d times its finite-difference operator (a = 1)
    are the assembled P1 mass and stiffness matrices."""
    M, K = element_assembly(dim, n)
    h = 1.0 / (n + 1)
    Mo = st.assemble_M(dim, [n] * dim, "p1").toarray() * h ** dim
    Ko = st.assemble_A(dim, [n] * dim, ONE, 0.0).toarray() * h ** dim
    assert np.abs(Mo - M).max() <= 1e-15
    assert np.abs(Ko - K).max() <= 1e-12 * np.abs(K).max()


def test_table1_matrices_are_the_p1_stencils():
    """The 1-D matrices behind the Table 1 pin (§8.1) are h times the P1 stencils used everywhere."""
    h = 1.0 / 64
    M, A = st.fem1d_matrices(h)
    assert np.abs(M - h * st.assemble_M(1, [63], "p1").toarray()).max() <= 1e-16
    assert np.abs(A - h * st.assemble_A(1, [63], ONE, 0.0).toarray()).max() <= 1e-10


@pytest.mark.parametrize("n,m,a0", [(31, 3, 0.7), (15, 1, 1.3)])
def test_p1_eigenmode_decay_closed_form_1d(n, m, a0):
    """1-D, constant a: sin(m pi x) is an eigenvector of the P1 mass (over h) with
    lambda_M = 2/3 + cos(m pi h)/3 and of A with lambda_A = 4 a0 h^-2 sin^2(m pi h / 2), so
    M (u_n - u_{n-1}) + tau A u_n = 0 gives u_n = (lambda_M / (lambda_M + tau lambda_A))^n u0."""
    p = S.eigenmode(1, n, 10, 0.4, a0, (m,))
    u0 = S.initial(p)
    u = oracle.implicit_euler(1, p.n, p.N, p.T, p.coeff, S.source(p), u0, mass="p1")
    h, tau = 1.0 / (n + 1), p.T / p.N
    lm = 2 / 3 + math.cos(m * math.pi * h) / 3
    la = 4 * a0 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2
    exact = np.stack([(lm / (lm + tau * la)) ** k * u0 for k in range(1, p.N + 1)])
    assert np.abs(u - exact).max() < 1e-13


@pytest.mark.parametrize("prob", [S.heat1d_mms(7, 8), S.heat2d_uniform(3, 6), S.heat2d_uniform(7, 3)],
                         ids=lambda p: p.name)
def test_p1_saddle_point_brute_force(prob):
    """Dense solve of eq. 2.7 with K (x) M reproduces the P1 time stepping, with p = -u."""
    p = prob
    f, u0 = S.source(p), S.initial(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, mass="p1")
    F = T.rhs(f, u0)
    sol = np.linalg.solve(st.dense_saddle(T), np.concatenate([-F.ravel(), -F.ravel()]))
    pp, uu = sol[: F.size].reshape(F.shape), sol[F.size:].reshape(F.shape)
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, u0, mass="p1")
    scale = np.abs(ref).max()
    assert np.abs(uu - ref).max() <= 1e-12 * scale
    assert np.abs(pp + ref).max() <= 1e-12 * scale
    # and B u = F through the C operator
    Bu = oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, ref, mass="p1")
    assert np.abs(Bu - F).max() <= 1e-13 * np.abs(F).max()


def test_p1_apply_B_matches_assembled():
    p = S.heat2d_uniform(7, 5)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, mass="p1")
    v = np.random.default_rng(0).standard_normal((p.N, p.ns))
    assert np.abs(oracle.apply_B(p.dim, p.n, p.N, p.T, p.coeff, v, mass="p1") - T.B(v)).max() < 1e-12


def test_p1_cg_agrees_with_cholesky():
    p = S.heat2d_uniform(15, 4)
    f = S.source(p)
    a = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, mass="p1")
    b = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, method="cg", cg_tol=1e-15, mass="p1")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def mms2d(n, N, T=1.0):
    """u = sin(pi x) sin(pi y) e^{-t} with the coefficient of the 2-D workload,
    a = 1 + 0.5 sin(2 pi x) sin(2 pi y) cos(2 pi t): f = u_t - div(a grad u) at the nodes."""
    p = S.heat2d_uniform(n, N)
    x, y = S.grid_axes(2, p.n)
    X, Y = np.meshgrid(x, y)  # rows y, columns x: x fastest when raveled
    f, ue = [], []
    for k in range(1, N + 1):
        t = k * T / N
        s = math.exp(-t)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y) * s
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) * s
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y) * s
        a = 1 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * math.cos(2 * np.pi * t)
        ax = np.pi * np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y) * math.cos(2 * np.pi * t)
        ay = np.pi * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * math.cos(2 * np.pi * t)
        f.append((-u - ax * ux - ay * uy + 2 * np.pi ** 2 * a * u).ravel())
        ue.append(u.ravel())
    u0 = (np.sin(np.pi * X) * np.sin(np.pi * Y)).ravel()
    return p, np.array(f), u0, np.array(ue)


def test_p1_mms_first_order_in_time_second_in_space_2d():
    """P1 in space, implicit Euler in time: the nodal error is O(tau + h^2); halving h and
    quartering tau divides it by about 4."""
    errs = []
    for n, N in [(15, 16), (31, 64)]:
        p, f, u0, ue = mms2d(n, N)
        u = oracle.implicit_euler(2, p.n, N, 1.0, p.coeff, f, u0, mass="p1")
        errs.append(np.abs(u - ue).max())
    assert 3.3 < errs[0] / errs[1] < 4.7, errs


@pytest.mark.parametrize("solver", ["exact", "vcycle"])
def test_p1_uzawa_converges_to_stepped_solution(solver):
    """The inexact Uzawa iteration (eq. 3.1) with H_k = mu_k M + tau A converges to the P1 stepped
    solution, with exact spatial solves and with the V-cycle reading."""
    p = S.heat2d_uniform(15, 8)
    f = S.source(p)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, mass="p1")
    F = T.rhs(f, None)
    if solver == "exact":
        Asolve, Hsolve = T.exact_A_solver(), T.exact_H_solver()
    else:
        Asolve, Hsolve = mg.st_vcycles(T)
    u, pp, hist = T.uzawa(F, 0.5, 400, Asolve, Hsolve, tol=1e-12)
    assert hist[-1] <= 1e-12
    ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f, mass="p1")
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-10


def test_p1_vcycle_for_H_is_symmetric_and_contracting():
    """The V-cycle of mu_k M + tau Abar stays a symmetric convergent approximation (eq. 4.7)."""
    p = S.heat2d_uniform(15, 4)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff, mass="p1")
    _, Hsolve = mg.st_vcycles(T, h_cycles=1)
    mus = st.mu(p.N)
    for k in (0, p.N - 1):
        V = np.stack([Hsolve(k, e) for e in np.eye(p.ns)], axis=1)
        assert np.abs(V - V.T).max() <= 1e-12 * np.abs(V).max()
        H = (mus[k] * T.M + T.tau * T.Abar).toarray()
        rho = np.abs(np.linalg.eigvals(np.eye(p.ns) - V @ H)).max()
        assert rho < 0.5
