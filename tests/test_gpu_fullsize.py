"""Parity at the full sizes of the workloads: the CUDA path (through the C ABI) against the oracle.

The time-global solution is the implicit-Euler solution (§2, eq. 2.1 and eq. 2.7), so the oracle
is sequential implicit Euler.  Where it finishes in minutes it runs over every step (the 2-D
workload, 255^2 x 1024, banded Cholesky); where it does not (the 3-D workload 127^3 x 256 needs CG
at tens of seconds per step, and the largest batch problems) it runs over the first steps, and
every step is covered by a rigorous a-posteriori bound computed from the oracle's B:

    with r = F - B u and e = u - u*,   e_n = (I + tau_n A_n)^-1 (e_{n-1} - r_n),  e_0 = 0,
    ||(I + tau_n A_n)^-1||_2 <= q_n = 1 / (1 + tau_n a_min lambda_min(L_h)),

because A_n >= a_min L_h in the SPD order (every face coefficient is at least a_min = a0 - |c|) and
lambda_min(L_h) = d (4/h^2) sin^2(pi h / 2); hence ||e_n|| <= q_n (||e_{n-1}|| + ||r_n||).
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64_TOL = 1e-10      # relative L2 vs the oracle for FP64 solves
MIXED_TOL = 1e-8      # relative L2 vs the oracle after refinement, mixed precision


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1802_08126_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def solve(prob, f, precision, tol, max_it=4000):
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, S.initial(prob), precision=precision,
                     omega=0.5) as P:
        u = np.zeros((prob.N, prob.ns))
        stt, it, hist = P.solve(tol, max_it, u_out=u)
    return stt, it, hist, u


def rel_err(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def rhs(prob, f):
    F = (prob.T / prob.N) * f
    u0 = S.initial(prob)
    if u0 is not None:
        F = F.copy()
        F[0] += u0.ravel()
    return F


def error_bound(prob, f, u):
    """Upper bound of ||u - u*|| / ||u*|| over all steps from the oracle's residual (module doc)."""
    r = rhs(prob, f)
    r -= oracle.apply_B(prob.dim, prob.n, prob.N, prob.T, prob.coeff, u)
    rn = np.linalg.norm(r, axis=1)
    h = 1.0 / (prob.n[0] + 1)
    lam = prob.dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a_min = prob.coeff.a0 - abs(prob.coeff.c)
    q = 1.0 / (1.0 + (prob.T / prob.N) * a_min * lam)
    e, acc = 0.0, 0.0
    for v in rn:
        e = q * (e + v)
        acc += e * e
    err = math.sqrt(acc)
    nu = np.linalg.norm(u)
    return err / max(nu - err, 1e-300), float(np.linalg.norm(r) / np.linalg.norm(rhs(prob, f)))


@pytest.fixture(scope="module")
def heat2d_full():
    """The 2-D workload (255^2, N_t = 1024, T = 1, f ~ U(-1,1) from seed 1) and its oracle solution
    over all 1024 steps (banded Cholesky per step)."""
    prob = S.heat2d_uniform(255, 1024)
    f = S.source(prob)
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f, None)
    return prob, f, ref


def test_heat2d_full_size_fp64_all_steps_match_oracle(heat2d_full):
    prob, f, ref = heat2d_full
    stt, it, hist, u = solve(prob, f, "fp64", 1e-12)
    assert stt == 0
    err = rel_err(u, ref)
    print("heat2d 255^2 x 1024 fp64: %d iterations, rel L2 vs oracle %.3e" % (it, err))
    assert err <= FP64_TOL


def test_heat2d_full_size_mixed_all_steps_match_oracle(heat2d_full):
    prob, f, ref = heat2d_full
    stt, it, hist, u = solve(prob, f, "mixed", 1e-11)
    assert stt == 0
    err = rel_err(u, ref)
    print("heat2d 255^2 x 1024 mixed: %d iterations, rel L2 vs oracle %.3e" % (it, err))
    assert err <= MIXED_TOL


def test_heat3d_full_size_mixed_matches_oracle():
    """The 3-D workload (127^3, N_t = 256, T = 2, mixed): the first steps against the oracle's
    implicit Euler with CG steps (relative residual 1e-14), and all 256 steps by the bound."""
    prob = S.heat3d_bumps(127, 256)
    f = S.source(prob)
    stt, it, hist, u = solve(prob, f, "mixed", 1e-10)
    assert stt == 0
    k = 3
    ref = oracle.implicit_euler(prob.dim, prob.n, prob.N, prob.T, prob.coeff, f[:k], S.initial(prob), steps=k,
                                method="cg", cg_tol=1e-14)
    err = rel_err(u[:k], ref)
    bound, res = error_bound(prob, f, u)
    print("heat3d 127^3 x 256 mixed: %d iterations, first %d steps rel L2 %.3e, all steps bound %.3e "
          "(oracle residual %.3e)" % (it, k, err, bound, res))
    assert err <= MIXED_TOL
    assert res <= 1e-10 * 1.01
    assert bound <= MIXED_TOL


# Batch workload: problem 96 has the strongest variation of the coefficient on the 255^2 grid
# (c = 0.80, alpha = 5), 309 the most steps on that grid (N_t = 1948), 30 the most steps with the
# smallest grid (31^2, N_t = 2003); 511 is 127^2 with 1987 steps.  They are solved together by
# pt_solve_batch in mixed precision, as the batch workload is.
BATCH_SAMPLE = [(96, None), (309, 48), (30, None), (511, 128)]


def test_batch_sample_matches_oracle():
    import paper_1802_08126_gb300 as ptu
    probs = [S.batch_problem(i) for i, _ in BATCH_SAMPLE]
    fs = [S.source(p) for p in probs]
    Ps = [ptu.Problem(p.dim, p.n, p.N, p.T, p.coeff, f, None, precision="mixed", omega=0.0) for p, f in zip(probs, fs)]
    try:
        its, sts = ptu.solve_batch(Ps, 1e-12, 6000)
        us = []
        for p, P in zip(probs, Ps):
            u = np.zeros((p.N, p.ns))
            P.get_state(u_out=u)
            us.append(u)
    finally:
        for P in Ps:
            P.close()
    for (i, k), p, f, u, it, stt in zip(BATCH_SAMPLE, probs, fs, us, its, sts):
        assert stt == 0, p.name
        steps = p.N if k is None else k
        ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, f[:steps], None, steps=steps)
        err = rel_err(u[:steps], ref)
        bound, res = error_bound(p, f, u)
        print("%s (c = %.3f): %d iterations, steps 1..%d rel L2 %.3e, all steps bound %.3e" %
              (p.name, p.coeff.c, it, steps, err, bound))
        assert err <= MIXED_TOL, p.name
        assert res <= 1e-12 * 1.01, p.name
        if k is not None:
            assert bound <= MIXED_TOL, p.name
