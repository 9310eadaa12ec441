"""Batched solves (one CUDA graph launch per iteration for many uneven problems), graph replay
versus plain launches, and the autotuner: all must return the same answers as solo solves."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1802_08126_gb300 import build
    build.build()


def make(prob, precision="fp64", **kw):
    import paper_1802_08126_gb300 as ptu
    return ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), S.initial(prob),
                       precision=precision, omega=0.5, **kw)


def state_u(P, prob):
    u = np.zeros((prob.N, prob.ns))
    P.get_state(u_out=u)
    return u


def test_batch_of_uneven_problems_equals_solo_solves():
    import paper_1802_08126_gb300 as ptu
    probs = [S.batch_problem(i) for i in range(6)]
    probs = [S.Problem(p.name, p.dim, [min(p.n[0], 63)] * 2, min(p.N, 300), p.T, p.coeff, p.f_kind, p.seed)
             for p in probs] + [S.heat1d_mms(31, 37), S.heat3d_bumps(7, 16)]
    precs = ["mixed", "fp64"] * (len(probs) // 2)
    solo = []
    for p, pr in zip(probs, precs):
        with make(p, pr) as P:
            st, it, _ = P.solve(1e-10, 600)
            solo.append((st, it, state_u(P, p)))
    Ps = [make(p, pr) for p, pr in zip(probs, precs)]
    its, sts = ptu.solve_batch(Ps, 1e-10, 600)
    for k, (p, P) in enumerate(zip(probs, Ps)):
        assert sts[k] == 0 and solo[k][0] == 0
        assert its[k] == solo[k][1], p.name
        u = state_u(P, p)
        assert np.array_equal(u, solo[k][2]), p.name
        ref = oracle.implicit_euler(p.dim, p.n, p.N, p.T, p.coeff, S.source(p), S.initial(p))
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-8
        P.close()


def test_batch_device_loop_matches_plain_launches_and_autotune_off():
    """The batch's device-side loop (one graph launch per quarter of the active set finishing),
    here with tuned launch configurations, gives the same iterates as the same batch untuned and
    solved by plain per-round launches of the same kernels, up to the rounding of the launch
    configuration."""
    import paper_1802_08126_gb300 as ptu
    probs = [S.batch_problem(i) for i in range(6, 12)]
    probs = [S.Problem(p.name, p.dim, [min(p.n[0], 63)] * 2, min(p.N, 300), p.T, p.coeff, p.f_kind, p.seed)
             for p in probs]
    out = []
    for kw, plain in ((dict(autotune=True), False), (dict(autotune=False), True)):
        Ps = [make(p, "mixed", **kw) for p in probs]
        ptu.profile_enable(plain)  # kernels timed one by one: the batch takes per-round host launches
        try:
            its, sts = ptu.solve_batch(Ps, 1e-10, 600)
        finally:
            ptu.profile_enable(False)
        assert all(s == 0 for s in sts)
        out.append((its, [state_u(P, p) for P, p in zip(Ps, probs)]))
        for P in Ps:
            P.close()
    for k, p in enumerate(probs):
        assert abs(out[0][0][k] - out[1][0][k]) <= 1, p.name
        assert np.linalg.norm(out[0][1][k] - out[1][1][k]) / np.linalg.norm(out[1][1][k]) <= 1e-9, p.name


def test_graph_replay_equals_plain_launches():
    prob = S.heat2d_uniform(31, 40)
    out = []
    for graphs in (True, False):
        with make(prob, graphs=graphs) as P:
            st, it, hist = P.solve(1e-11, 500)
            out.append((it, hist.copy(), state_u(P, prob)))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_configuration_gives_the_same_solution(precision, tmp_path, monkeypatch):
    monkeypatch.setenv("PT_TUNE_CACHE", str(tmp_path / "tune.json"))
    prob = S.heat2d_uniform(63, 48)
    with make(prob, precision) as P:
        P.solve(1e-10, 500)
        base = state_u(P, prob)
    with make(prob, precision, autotune=True) as P:
        st, it, _ = P.solve(1e-10, 500)
        tuned = state_u(P, prob)
    assert st == 0
    assert np.linalg.norm(tuned - base) / np.linalg.norm(base) <= (1e-12 if precision == "fp64" else 1e-9)
    for cols, ce in [(1, 256), (4, 4096), (16, 0)]:
        with make(prob, precision, dst_cols=cols, coarse_elems=ce) as P:
            st, it, _ = P.solve(1e-10, 500)
            u = state_u(P, prob)
        assert st == 0
        assert np.linalg.norm(u - base) / np.linalg.norm(base) <= (1e-12 if precision == "fp64" else 1e-9)


def test_device_generated_source_matches_host_generator():
    """pt_problem_set_rhs_uniform draws the same SplitMix64 field on the device as the host
    generator: the solutions agree bit for bit."""
    prob = S.heat2d_uniform(31, 20, seed=0x1234ABCD5678)
    with make(prob) as P:
        P.solve(1e-11, 500)
        u1 = state_u(P, prob)
        P.set_rhs_uniform(prob.seed)
        P.solve(1e-11, 500)
        u2 = state_u(P, prob)
    assert np.array_equal(u1, u2)


def test_default_omega_rule():
    """omega <= 0 selects 1.5 / (1 + alpha); for |c| = a0 / 2 that is the 0.5 used elsewhere."""
    prob = S.heat2d_uniform(15, 16)
    import paper_1802_08126_gb300 as ptu
    out = []
    for om in (0.0, 0.5):
        with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), None, omega=om) as P:
            st, it, hist = P.solve(1e-10, 500)
            out.append(hist.copy())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dim,n,N,precision", [(2, 255, 64, "mixed"), (2, 255, 64, "fp64"), (2, 31, 300, "mixed"),
                                               (3, 31, 16, "mixed"), (3, 15, 8, "fp64"), (1, 63, 64, "fp64")])
def test_memory_estimate_covers_the_allocation(dim, n, N, precision):
    """The admission estimate (serving loop, batch waves) is an upper bound of what a problem
    actually allocates."""
    import paper_1802_08126_gb300 as ptu
    from synthetic import Coeff
    coeff = Coeff(a0=1.0, c=0.5, fx=[S.TRIG_SIN] * 3, mx=[2.0] * 3, ft=S.TRIG_COS, mt=2.0)  # mean-zero in t
    solver = "exact" if dim == 1 else "mg"
    P = ptu.Problem(dim, [n] * dim, N, 1.0, coeff, None, None, precision=precision, solver=solver)
    try:
        held = P.device_bytes()
    finally:
        P.close()
    est = ptu.estimate_bytes(dim, [n] * dim, N, precision, solver=solver)
    assert held <= est, (held, est)
