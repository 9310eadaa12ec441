import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer-running CPU check")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def sine_H_solver(T):
    """A second exact solver of H_k = mu_k I + tau Abar for a reference coefficient a0 constant in
    space (finite differences, uniform grid): the sine transform of type I diagonalises the
    Dirichlet Laplacian, eigenvalues (4/h^2) sin^2(pi k h / 2) per axis.  It needs no
    factorisation, so it reaches grids where the sparse direct solver of the oracle is too slow;
    tests/test_oracle_spectral.py checks it against that solver on small grids."""
    import numpy as np
    import scipy.fft as sf
    from oracle.spacetime import mu
    n, dim = T.n[0], T.dim
    h = 1.0 / (n + 1)
    lam1 = 4.0 / (h * h) * np.sin(np.pi * np.arange(1, n + 1) * h / 2.0) ** 2
    lam = np.zeros((n,) * dim)
    for d in range(dim):
        shape = [1] * dim
        shape[d] = n
        lam = lam + lam1.reshape(shape)
    lam *= T.coeff.a0
    m = mu(T.N)

    def solve(k, r):
        rs = np.asarray(r).reshape((n,) * dim)
        c = sf.dstn(rs, type=1, norm="ortho") / (m[k] + T.tau * lam)
        return sf.dstn(c, type=1, norm="ortho").reshape(-1)
    return solve
