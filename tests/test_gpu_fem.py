"""The P1 finite-element form (M != I in §2, eq. 2.1) on the GPU, through the C ABI: the operator B,
the Schur complement S, the preconditioner H~^-1 and full solves against the oracle; Table 1 of
§8.1 (extremal eigenvalues of H^-1 S) by a Lanczos iteration built on the library's S and H^-1;
and the setting of Table 2 (§8.2: iterations to a 1e-6 relative error in the S-norm)."""
import math
import types

import numpy as np
import pytest

import oracle
import synthetic as S
from tests.conftest import read_golden
from oracle import mg
from oracle import spacetime as st

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ONE = types.SimpleNamespace(a0=1.0, c=0.0, fx=[0, 0, 0], mx=[0.0] * 3, ft=0, mt=0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1802_08126_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def problem(prob, coeff=None, solver="mg", **kw):
    import paper_1802_08126_gb300 as ptu
    coeff = prob.coeff if coeff is None else coeff
    return ptu.Problem(prob.dim, prob.n, prob.N, prob.T, coeff, S.source(prob), S.initial(prob), precision="fp64",
                       solver=solver, mass="p1", **kw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [S.heat1d_mms(15, 8), S.heat2d_uniform(7, 6), S.heat2d_uniform(31, 4), S.heat2d_uniform(63, 3),
         S.heat2d_uniform(127, 2)]


@pytest.mark.parametrize("prob", CASES, ids=lambda p: p.name)
def test_p1_apply_B_matches_oracle(prob):
    u = np.random.default_rng(1).standard_normal((prob.N, prob.ns))
    with problem(prob) as P:
        out = torch.empty_like(dev(u))
        P.apply_B(dev(u), out)
    ref = oracle.apply_B(prob.dim, prob.n, prob.N, prob.T, prob.coeff, u, mass="p1")
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prob", [S.heat1d_mms(15, 8), S.heat1d_mms(63, 16)], ids=lambda p: p.name)
def test_p1_exact_1d_preconditioners_and_schur_complement(prob):
    """1-D exact solves: A~ = A, H~_k = H_k = mu_k M + tau Abar (tridiagonal), and S = K^T A^-1 K +
    K + K^T + A with K = K (x) M (eq. 2.5) against the assembled oracle operators."""
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, mass="p1")
    r = np.random.default_rng(2).standard_normal((prob.N, prob.ns))
    with problem(prob, solver="exact") as P:
        out = torch.empty_like(dev(r))
        P.precond_H(dev(r), out)
        assert rel(host(out), T.apply_Hinv(r, T.exact_H_solver())) <= 1e-11
        P.precond_A(dev(r), out)
        Asol = T.exact_A_solver()
        assert rel(host(out), Asol(r)) <= 1e-11
        P.apply_S(dev(r), out)
        ref = T.Kt(Asol(T.K(r))) + T.K(r) + T.Kt(r) + T.Ablk(r)
        assert rel(host(out), ref) <= 1e-11


@pytest.mark.parametrize("prob", [S.heat2d_uniform(15, 8), S.heat2d_uniform(63, 3)], ids=lambda p: p.name)
@pytest.mark.parametrize("cycles", [1, 2])
def test_p1_vcycle_H_matches_oracle_vcycle(prob, cycles):
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, mass="p1")
    _, Hsolve = mg.st_vcycles(T, h_cycles=cycles)
    r = np.random.default_rng(3).standard_normal((prob.N, prob.ns))
    with problem(prob, n_vcycles=cycles) as P:
        out = torch.empty_like(dev(r))
        P.precond_H(dev(r), out)
    assert rel(host(out), T.apply_Hinv(r, Hsolve)) <= 1e-11


@pytest.mark.parametrize("prob,solver", [(S.heat1d_mms(31, 16), "exact"), (S.heat2d_uniform(15, 16), "mg"),
                                         (S.heat2d_uniform(63, 32), "mg")], ids=lambda v: getattr(v, "name", v))
def test_p1_solve_matches_oracle_stepping(prob, solver):
    f, u0 = S.source(prob), S.initial(prob)
    with problem(prob, solver=solver, omega=0.5) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(1e-12, 2000, u_out=u)
    assert stt == 0
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, u0, mass="p1")
    assert rel(u, ref) <= 1e-10


def test_p1_history_mirrors_oracle_uzawa():
    prob = S.heat2d_uniform(15, 8)
    T = st.SpaceTime(prob.dim, prob.n, prob.N, prob.T, prob.coeff, mass="p1")
    F = T.rhs(S.source(prob), None)
    Asolve, Hsolve = mg.st_vcycles(T)
    _, _, hist_ref = T.uzawa(F, 0.5, 12, Asolve, Hsolve)
    with problem(prob, omega=0.5, h_solver="vcycle") as P:
        _, it, hist = P.solve(0.0, 12)
    assert it == 12
    assert np.abs(hist - hist_ref).max() <= 1e-9 * hist_ref.max()


def lanczos_extremes(P, N, ns, iters, seed=0):
    """Extremal eigenvalues of H^-1 S (the pencil S v = lambda H v) by the Lanczos process with
    H-orthonormal vectors q_j (p_j = H q_j), full reorthogonalisation, using the library's S and
    H^-1: w = S q_j - alpha p_j - beta p_{j-1}, q_{j+1} = H^-1 w / beta."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    r = torch.randn((N, ns), dtype=torch.float64, device="cuda", generator=g)
    z = torch.empty_like(r)
    P.precond_H(r, z)
    b = math.sqrt(float((r * z).sum()))
    Q, Pv, al, be = [z / b], [r / b], [], []
    w = torch.empty_like(r)
    for _ in range(iters):
        P.apply_S(Q[-1], w)
        a = float((Q[-1] * w).sum())
        al.append(a)
        w -= a * Pv[-1]
        if be:
            w -= be[-1] * Pv[-2]
        for _ in range(2):
            for q, p in zip(Q, Pv):
                w -= float((q * w).sum()) * p
        P.precond_H(w, z)
        bb = math.sqrt(float((w * z).sum()))
        be.append(bb)
        Q.append(z / bb)
        Pv.append(w / bb)
    Tm = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    e = np.linalg.eigvalsh(Tm)
    return e[0], e[-1]


TABLE1 = [(int(r[0]), int(r[1]), float(r[2]), float(r[3])) for r in read_golden("table1.txt")]


@pytest.mark.parametrize("hinv,N,lmin,lmax", [t for t in TABLE1 if t[1] in (4, 16, 64, 256, 1024)],
                         ids=lambda v: str(v))
def test_table1_extremal_eigenvalues_on_gpu(hinv, N, lmin, lmax):
    """Table 1 of §8.1: 1-D heat equation, P1 in space, T = 1, uniform steps, exact spatial solves
    (alpha = 1); the library's H^-1 S has the printed extremal eigenvalues (4 decimals)."""
    n = hinv - 1
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(1, [n], N, 1.0, ONE, None, None, precision="fp64", solver="exact", mass="p1") as P:
        lo, hi = lanczos_extremes(P, N, n, 250)
    assert abs(lo - lmin) <= 6e-5, (lo, lmin)
    assert abs(hi - lmax) <= 6e-5, (hi, lmax)


def table2_iterations(n, N, omega=0.9, max_it=80):
    """The setting of Table 2 (§8.2): 2-D, P1, a = 1, T = 1, u(0) = sin(pi x) sin(pi y), f = 0, one
    V-cycle for A~ and for H~, omega = 0.9; the first j with ||u - u_j||_S < 1e-6 ||u||_S, the S-norm
    (eq. 2.5, exact A) and u from the oracle."""
    import paper_1802_08126_gb300 as ptu
    T = st.SpaceTime(2, [n, n], N, 1.0, ONE, mass="p1")
    u0 = S.sin_mode(2, [n, n], (1, 1))
    ustar = oracle.implicit_euler(2, [n, n], N, 1.0, ONE, np.zeros((N, T.ns)), u0, mass="p1")
    import scipy.sparse.linalg as spla
    lu = spla.splu((T.tau * T.A[0]).tocsc())

    def snorm(e):
        Ke = T.K(e)
        z = lu.solve(np.ascontiguousarray(Ke.T)).T
        return math.sqrt(np.sum(Ke * z) + 2 * np.sum(e * Ke) + np.sum(e * T.Ablk(e)))

    ref = snorm(ustar)
    with ptu.Problem(2, [n, n], N, 1.0, ONE, None, u0, precision="fp64", omega=omega, n_vcycles=1,
                     h_solver="vcycle", mass="p1") as P:
        u = np.zeros((N, T.ns))
        for j in range(15, max_it):
            P.solve(0.0, j, u_out=u)
            if snorm(u - ustar) < 1e-6 * ref:
                return j
    return None


def test_table2_setting_iterations_flat_in_h_and_N():
    """Table 2 prints 20-22 iterations for h = 1/8 .. 1/64 and N = 128 .. 1024.  With this library's
    V-cycle reading the counts differ from the printed ones by a few iterations; the claim tested
    is the paper's: they stay flat in h and N."""
    counts = {}
    for hinv in (8, 16, 32, 64):
        for N in (128, 1024):
            counts[(hinv, N)] = table2_iterations(hinv - 1, N)
    print("Table 2 setting (h^-1, N) -> iterations:", counts)
    vals = list(counts.values())
    assert all(v is not None for v in vals)
    assert max(vals) - min(vals) <= 3
    assert max(vals) <= 30
