"""The paper's central claim in the form this implementation can check (§8.2, Table 2, in
character): the number of Uzawa iterations to a fixed tolerance does not grow with the number
of time steps N_t, so the time-global solve costs O(N_t) work per iteration and a flat number
of iterations.  2-D family 127^2 (exact and V-cycle H_k solves) and the 1-D family with exact
spatial solves."""
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _iterations(prob, **kw):
    import paper_1802_08126_gb300 as ptu
    with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, None, None, **kw) as P:
        P.set_rhs_uniform(prob.seed)
        st, it, _ = P.solve(1e-8, 1000)
    assert st == 0
    return it


@pytest.mark.parametrize("h_solver", ["exact", "vcycle"])
def test_iterations_flat_in_nt_2d(h_solver):
    its = [_iterations(S.heat2d_uniform(127, N), precision="fp64", omega=0.5, h_solver=h_solver)
           for N in (64, 256, 1024, 2048)]
    assert max(its) - min(its) <= max(3, 0.1 * max(its)), its


def test_iterations_flat_in_nt_1d_exact_solves():
    its = []
    for N in (16, 64, 256, 1024):
        prob = S.heat1d_mms(63, N)
        import paper_1802_08126_gb300 as ptu
        with ptu.Problem(prob.dim, prob.n, prob.N, prob.T, prob.coeff, S.source(prob), S.initial(prob),
                         precision="fp64", omega=0.5, solver="exact") as P:
            st, it, _ = P.solve(1e-8, 1000)
        assert st == 0
        its.append(it)
    assert max(its) - min(its) <= max(3, 0.1 * max(its)), its
