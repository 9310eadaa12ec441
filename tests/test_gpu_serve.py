"""Serving loop: continuous batching with HBM admission.  Each served result must equal the result
of solving the same problem alone, whatever else was on the device at the time."""
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


def solo(prob, precision="mixed", tol=1e-9):
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, None, S.initial(prob),
                     precision=precision) as P:
        P.set_rhs_uniform(prob.seed, S.initial(prob)) if prob.f_kind == "uniform" else P.set_rhs(S.source(prob), S.initial(prob))
        st, it, _ = P.solve(tol, 2000)
        u = np.zeros((prob.N, prob.ns))
        P.get_state(u_out=u)
    return st, it, u


def submit(sv, prob, precision="mixed", tol=1e-9):
    if prob.f_kind == "uniform":
        return sv.submit(prob.dim, prob.n, prob.N, prob.T, prob.coeff, None, seed=prob.seed, u0=S.initial(prob),
                         tol=tol, precision=precision)
    return sv.submit(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), u0=S.initial(prob), tol=tol,
                     precision=precision)


def workload():
    out = []
    for i in range(5):
        p = S.batch_problem(i)
        out.append(S.Problem(p.name, 2, [min(p.n[0], 63)] * 2, min(p.N, 200), p.T, p.coeff, "uniform", p.seed))
    out.append(S.heat1d_mms(63, 64))
    out.append(S.heat3d_bumps(7, 12))
    return out


def test_results_are_the_same_alone_and_in_the_mix():
    import paper_1802_08126_gb300 as ptu
    probs = workload()
    ref = [solo(p) for p in probs]
    with ptu.Server() as sv:
        tickets = [submit(sv, p) for p in probs]
        for p, t, (st0, it0, u0) in zip(probs, tickets, ref):
            u = np.zeros((p.N, p.ns))
            st, it = sv.wait(t, u)
            assert st == 0 and st0 == 0
            assert it == it0, p.name
            assert np.array_equal(u, u0), p.name
        stats = sv.stats()
    assert stats["completed"] == len(probs)
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    assert stats["dofs_per_s"] > 0


def test_requests_arriving_while_others_run_are_admitted():
    """Continuous batching: later requests join while an earlier, longer solve is still running,
    finish before it, and still give their stand-alone answers."""
    import paper_1802_08126_gb300 as ptu
    big = S.heat2d_uniform(255, 1024)
    small = workload()[:3]
    ref_big = solo(big, tol=1e-10)
    ref_small = [solo(p) for p in small]
    with ptu.Server() as sv:
        tb = submit(sv, big, tol=1e-10)
        with pytest.raises(ptu.PtError) as e:
            sv.wait(tb, timeout_ms=0)   # running: a bounded wait returns PT_ETIMEOUT
        assert e.value.status == 6
        ts = [submit(sv, p) for p in small]
        for p, t, (st0, it0, u0) in zip(small, ts, ref_small):
            u = np.zeros((p.N, p.ns))
            assert sv.wait(t, u) == (0, it0)
            assert np.array_equal(u, u0)
        with pytest.raises(ptu.PtError):
            sv.wait(tb, timeout_ms=0)   # the small ones finished while the big one still runs
        u = np.zeros((big.N, big.ns))
        assert sv.wait(tb, u) == (0, ref_big[1])
        assert np.array_equal(u, ref_big[2])
    f = oracle.implicit_euler(2, big.n, big.N, big.T, big.coeff, S.source(big), None, steps=2)
    assert np.linalg.norm(u[:2] - f) / np.linalg.norm(f) <= 1e-8


def test_admission_rejects_requests_beyond_the_budget():
    import paper_1802_08126_gb300 as ptu
    prob = S.heat2d_uniform(255, 1024)
    with ptu.Server(hbm_budget=64 << 20) as sv:
        with pytest.raises(ptu.PtError) as e:
            submit(sv, prob)
        assert e.value.status == 2  # PT_ENOMEM, decided on the host before any device work
