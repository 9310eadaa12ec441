"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the solver: it only defines the problem
instances (grids, step counts, coefficient parameters) and generates their
source terms and initial data from fixed seeds.  Both the oracle and the GPU
path receive the arrays produced here; neither side imports the other.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``seed`` is the ``(i+1)``-th output of the
generator started at state ``seed``.  A double in [0, 1) takes the top 53 bits.

Array layout everywhere: ``[N_t][n_z][n_y][n_x]`` with x fastest, interior grid
points only, point ``i`` of an axis at ``x = (i + 1) h``, ``h = 1/(n + 1)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TRIG_ONE, TRIG_SIN, TRIG_COS = 0, 1, 2


def splitmix64(seed: int, index) -> np.ndarray:
    """Output ``index`` (0-based, array-like) of SplitMix64 started at ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits of the SplitMix64 draws."""
    z = splitmix64(seed, index)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, count: int, offset: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """``count`` i.i.d. U(-1,1) values (2 U[0,1) - 1), draws offset..offset+count-1."""
    out = np.empty(count, dtype=np.float64)
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        out[s:e] = 2.0 * uniform01(seed, np.arange(offset + s, offset + e, dtype=np.uint64)) - 1.0
    return out


@dataclasses.dataclass
class Coeff:
    """a(x,t) = a0 + c * prod_d g_d(pi*mx[d]*x_d) * g_t(pi*mt*t), g in {1, sin, cos}."""

    a0: float = 1.0
    c: float = 0.0
    fx: Sequence[int] = (TRIG_ONE, TRIG_ONE, TRIG_ONE)
    mx: Sequence[float] = (0.0, 0.0, 0.0)
    ft: int = TRIG_ONE
    mt: float = 0.0


@dataclasses.dataclass
class Problem:
    """One time-global heat problem u_t - div(a grad u) = f on the unit box."""

    name: str
    dim: int
    n: Sequence[int]
    N: int
    T: float
    coeff: Coeff
    f_kind: str  # "uniform", "mms1", "bumps", "zero"
    seed: int = 0
    u0_kind: str = "zero"  # "zero" or "mms1" or "sinmode"
    n_bumps: int = 8
    sigma: float = 0.1
    mode: Sequence[int] = (1, 1, 1)
    taus: Optional[np.ndarray] = None  # step lengths tau_1..tau_N, None: uniform T/N

    @property
    def ns(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    @property
    def dofs(self) -> int:
        return self.ns * self.N


def grid_axes(dim: int, n: Sequence[int]):
    """Interior node coordinates per axis."""
    return [np.arange(1, n[d] + 1, dtype=np.float64) / (n[d] + 1) for d in range(dim)]


def _mesh(dim: int, n: Sequence[int]):
    axes = grid_axes(dim, n)
    # meshgrid with x fastest in memory: arrays shaped [n_z][n_y][n_x]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]  # x, y, z in that order


def random_steps(N: int, T: float, seed: int, spread: float = 0.5) -> np.ndarray:
    """Quasi-uniform step lengths tau_n = T w_n / sum(w), w_n = 1 + spread U_n, U_n = draw n-1
    of SplitMix64(seed): the ratio of any two steps is at most 1 + spread."""
    w = 1.0 + spread * uniform01(seed, np.arange(N, dtype=np.uint64))
    return T * w / w.sum()


def times(N: int, T: float, taus: Optional[np.ndarray] = None) -> np.ndarray:
    """t_1..t_N: n T/N, or the partial sums of the given step lengths."""
    if taus is None:
        return np.arange(1, N + 1) * (T / N)
    return np.cumsum(np.asarray(taus, dtype=np.float64))


def mms1_exact(n: int, N: int, T: float, taus: Optional[np.ndarray] = None) -> np.ndarray:
    """Manufactured solution u = sin(pi x) exp(-t) at (x_i, t_n), n = 1..N."""
    x = grid_axes(1, [n])[0]
    t = times(N, T, taus)
    return np.exp(-t)[:, None] * np.sin(math.pi * x)[None, :]


def mms1_f(n: int, N: int, T: float, taus: Optional[np.ndarray] = None) -> np.ndarray:
    """Source for u = sin(pi x) e^{-t}, a = 1 + 0.5 sin(pi x) cos(2 pi t) in 1-D."""
    x = grid_axes(1, [n])[0][None, :]
    t = times(N, T, taus)[:, None]
    a = 1.0 + 0.5 * np.sin(math.pi * x) * np.cos(2 * math.pi * t)
    ax = 0.5 * math.pi * np.cos(math.pi * x) * np.cos(2 * math.pi * t)
    return np.exp(-t) * (-np.sin(math.pi * x) - math.pi * ax * np.cos(math.pi * x)
                         + math.pi ** 2 * a * np.sin(math.pi * x))


def bump_centres(seed: int, count: int, dim: int) -> np.ndarray:
    return uniform01(seed, np.arange(count * dim, dtype=np.uint64)).reshape(count, dim)


def bumps_field(dim: int, n: Sequence[int], seed: int, count: int, sigma: float) -> np.ndarray:
    """sum_i exp(-|x - c_i|^2 / (2 sigma^2)) on the interior grid, centres U(0,1)^dim."""
    xs = _mesh(dim, n)
    cs = bump_centres(seed, count, dim)
    out = np.zeros(xs[0].shape)
    for c in cs:
        r2 = sum((xs[d] - c[d]) ** 2 for d in range(dim))
        out += np.exp(-r2 / (2 * sigma * sigma))
    return out.reshape(-1)


def sin_mode(dim: int, n: Sequence[int], mode: Sequence[int]) -> np.ndarray:
    xs = _mesh(dim, n)
    out = np.ones(xs[0].shape)
    for d in range(dim):
        out = out * np.sin(math.pi * mode[d] * xs[d])
    return out.reshape(-1)


def source(p: Problem, steps: Optional[int] = None) -> np.ndarray:
    """f(x_i, t_n) for n = 1..steps (default N), shape [steps][ns]."""
    steps = p.N if steps is None else steps
    if p.f_kind == "uniform":
        return uniform_pm1(p.seed, steps * p.ns).reshape(steps, p.ns)
    if p.f_kind == "mms1":
        return mms1_f(p.n[0], p.N, p.T, p.taus)[:steps]
    if p.f_kind == "bumps":
        b = bumps_field(p.dim, p.n, p.seed, p.n_bumps, p.sigma)
        return np.broadcast_to(b, (steps, p.ns)).copy()
    if p.f_kind == "zero":
        return np.zeros((steps, p.ns))
    raise ValueError(p.f_kind)


def initial(p: Problem) -> Optional[np.ndarray]:
    if p.u0_kind == "zero":
        return None
    if p.u0_kind == "mms1":
        return np.sin(math.pi * grid_axes(1, p.n)[0])
    if p.u0_kind == "sinmode":
        return sin_mode(p.dim, p.n, p.mode)
    raise ValueError(p.u0_kind)


# ---- the workloads -------------------------------------------------------------

def heat1d_mms(n: int = 63, N: int = 64) -> Problem:
    """1-D heat, a = 1 + 0.5 sin(pi x) cos(2 pi t), manufactured u = sin(pi x) e^{-t}, T = 1."""
    return Problem("heat1d_mms_n%d_N%d" % (n, N), 1, [n], N, 1.0,
                   Coeff(1.0, 0.5, (TRIG_SIN, TRIG_ONE, TRIG_ONE), (1.0, 0, 0), TRIG_COS, 2.0),
                   "mms1", u0_kind="mms1")


def heat2d_uniform(n: int = 255, N: int = 1024, seed: int = 1) -> Problem:
    """2-D heat, a = 1 + 0.5 sin(2 pi x) sin(2 pi y) cos(2 pi t), f ~ U(-1,1), u0 = 0, T = 1."""
    return Problem("heat2d_n%d_N%d" % (n, N), 2, [n, n], N, 1.0,
                   Coeff(1.0, 0.5, (TRIG_SIN, TRIG_SIN, TRIG_ONE), (2.0, 2.0, 0), TRIG_COS, 2.0),
                   "uniform", seed=seed)


def heat3d_bumps(n: int = 127, N: int = 256, seed: int = 3) -> Problem:
    """3-D heat, a = 1 + 0.5 cos(2pi x)cos(2pi y)cos(2pi z) sin(pi t), 8 Gaussian bumps, T = 2."""
    return Problem("heat3d_n%d_N%d" % (n, N), 3, [n, n, n], N, 2.0,
                   Coeff(1.0, 0.5, (TRIG_COS, TRIG_COS, TRIG_COS), (2.0, 2.0, 2.0), TRIG_SIN, 1.0),
                   "bumps", seed=seed, n_bumps=8, sigma=0.1)


def batch_problem(i: int, master_seed: int = 4) -> Problem:
    """Problem i of the 512-problem batch: all parameters from SplitMix64(master_seed) draws 16i..16i+15."""
    u = uniform01(master_seed, np.arange(16 * i, 16 * i + 8, dtype=np.uint64))
    n = (31, 63, 127, 255)[min(3, int(u[0] * 4))]
    N = int(round(math.exp(math.log(16) + u[1] * (math.log(2048) - math.log(16)))))
    c = 0.8 * float(u[2])
    kx = 1 + min(3, int(u[3] * 4))
    ky = 1 + min(3, int(u[4] * 4))
    fseed = int(splitmix64(master_seed, 16 * i + 8))
    return Problem("batch%d_n%d_N%d" % (i, n, N), 2, [n, n], N, 1.0,
                   Coeff(1.0, c, (TRIG_SIN, TRIG_SIN, TRIG_ONE), (2.0 * kx, 2.0 * ky, 0), TRIG_COS, 2.0),
                   "uniform", seed=fseed)


def eigenmode(dim: int, n: int, N: int, T: float, a0: float, mode: Sequence[int]) -> Problem:
    """Constant coefficient a0, f = 0, u0 = prod_d sin(m_d pi x_d)."""
    return Problem("mode%dd_n%d_N%d" % (dim, n, N), dim, [n] * dim, N, T,
                   Coeff(a0, 0.0), "zero", u0_kind="sinmode", mode=list(mode))
