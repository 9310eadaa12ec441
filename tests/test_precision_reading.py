"""The measurement behind the reading on BF16 storage (mixed precision): BF16 storage of the
smoother's vectors (every vector the A~ V-cycle writes) and of the Schur preconditioner's input
and output, emulated on the oracle's Uzawa iteration (§3, eq. 3.1) with FP64 outer residuals.
No GPU; the oracle itself stays FP64."""
import numpy as np

import synthetic as S
from oracle import mg
from oracle import spacetime as st


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as FP64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class StoredV(mg.VCycle):
    """The oracle's V-cycle with every stored vector passed through `rnd`."""

    def __init__(self, *args, rnd=None, **kw):
        super().__init__(*args, **kw)
        self.rnd = rnd

    def _cycle(self, l, b, rhs):
        L = self.L[l][b]
        if l == len(self.sizes) - 1:
            return self.rnd(rhs / L.diagonal())
        Dinv = self.Dinv[l][b]
        x = self.rnd(self.w * Dinv * rhs)
        rc = self.rnd((self.P[l].T @ (rhs - L @ x)) / (2 ** self.dim))
        x = self.rnd(x + self.P[l] @ self._cycle(l + 1, b, rc))
        return self.rnd(x + self.w * Dinv * (rhs - L @ x))


def test_bf16_rounding_is_round_to_nearest_even():
    """8 significant bits: the ulp at 1 is 2^-7, halfway cases go to the even significand."""
    x = np.array([1.0, -3.0, 1e-3, 123.456, 2.0 ** -20])
    assert np.all(np.abs(bf16(x) - x) <= 2.0 ** -8 * np.abs(x))
    assert bf16(1.0 + 2.0 ** -8) == 1.0
    assert bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7


def test_bf16_smoother_storage_keeps_the_iteration_count():
    """2-D workload family at 31^2 x 32: FP64, and BF16-stored smoother vectors with the H~ input
    and output rounded too, reach 1e-8 in the same number of iterations (52)."""
    p = S.heat2d_uniform(31, 32)
    T = st.SpaceTime(p.dim, p.n, p.N, p.T, p.coeff)
    F = T.rhs(S.source(p), None)
    Hs = T.exact_H_solver()
    build = lambda m: [T.taus[i] * st.assemble_A(2, [m, m], p.coeff, T.times[i]) for i in range(p.N)]
    its = {}
    for name, rnd in (("fp64", lambda a: a), ("bf16", bf16)):
        V = StoredV(2, p.n[0], build, rnd=rnd)
        plain = T.apply_Hinv
        T.apply_Hinv = lambda r, H: rnd(plain(rnd(r), H))
        try:
            _, _, hist = T.uzawa(F, 0.5, 200, V.apply, Hs, tol=1e-8)
        finally:
            T.apply_Hinv = plain
        assert hist[-1] <= 1e-8
        its[name] = len(hist) - 1
    assert abs(its["bf16"] - its["fp64"]) <= 1, its
