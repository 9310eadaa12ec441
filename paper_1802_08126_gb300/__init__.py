"""GB300-native time-parallel inexact Uzawa solver for parabolic problems.

Python binding of the C ABI in ``include/pt.h``: argument marshalling only, every step of the
solver runs in the CUDA library ``_lib/libptuzawa.so`` (built by ``build.build()``).  PyTorch is
used only to hold device memory and to name streams.

Method (Neumüller & Smears, "Time-parallel iterative solvers for parabolic evolution
equations"): implicit Euler over all N_t steps at once (§2, eq. 2.1-2.4), rewritten as the
symmetric saddle-point system of eq. 2.7 and solved by the inexact Uzawa iteration of §3,
eq. 3.1 with the DST-in-time Schur-complement preconditioner of §4, eq. 4.4-4.6.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import PT_EDIVERGED, PT_ENOTCONV, PT_OK  # noqa: F401

__all__ = ["Problem", "PtError", "launch_count", "status_name", "profile_enable", "profile_reset",
           "profile_totals", "dst_forward_noalloc", "solve_batch", "Server"]


class PtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (status_name(status), msg))
        self.status = status


def status_name(status: int) -> str:
    return _lib.load().pt_status_string(int(status)).decode()


def _check(status: int, allowed=(PT_OK,)):
    if status not in allowed:
        raise PtError(status, _lib.load().pt_last_error().decode())
    return status


def launch_count() -> int:
    """Kernel launches issued by the library so far (all problems)."""
    return int(_lib.load().pt_kernel_launch_count())


def profile_enable(on: bool = True) -> None:
    """Record CUDA-event timings of every later kernel launch (per kernel name)."""
    _lib.load().pt_profile_enable(1 if on else 0)


def profile_reset() -> None:
    _lib.load().pt_profile_reset()


def profile_totals() -> dict:
    """{kernel name: {"ms", "bytes", "flops", "launches"}} accumulated since the last reset."""
    L = _lib.load()
    count = L.pt_profile_get(-1, None, 0, None, None, None, None)
    out = {}
    for k in range(count):
        name = ctypes.create_string_buffer(64)
        ms, b, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_ulonglong()
        if L.pt_profile_get(k, name, 64, ctypes.byref(ms), ctypes.byref(b), ctypes.byref(fl), ctypes.byref(n)) < 0:
            break
        out[name.value.decode()] = {"ms": ms.value, "bytes": b.value, "flops": fl.value, "launches": n.value}
    return out


def _step_array(taus, N: int):
    """Host FP64 copy of the N step lengths (kept alive by the caller while the C call runs)."""
    if taus is None:
        return None
    a = np.ascontiguousarray(np.asarray(taus, dtype=np.float64).reshape(-1))
    if a.size != N:
        raise ValueError("need %d step lengths, got %d" % (N, a.size))
    return a


def _options(precision="mixed", omega=0.0, solver="mg", check_every=0, autotune=0, h_solver="auto",
             steps=None):
    o = _lib.Options()
    if steps is not None:
        o.tau_steps = steps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.h_solver = {"auto": 0, "vcycle": 1, "exact": 2}[h_solver]
    o.precision = {"fp64": _lib.PT_PREC_FP64, "mixed": _lib.PT_PREC_MIXED}[precision]
    o.omega = float(omega)
    o.spatial_solver = {"mg": _lib.PT_SOLVER_MG, "exact": _lib.PT_SOLVER_EXACT_1D}[solver]
    o.check_every = int(check_every)
    o.autotune = 1 if autotune is True else (-1 if autotune is False else int(autotune))
    return o


def estimate_bytes(dim: int, n: Sequence[int], N: int, precision: str = "mixed", solver: str = "mg") -> int:
    """Upper estimate of the device memory a problem of this size takes (no allocation)."""
    L = _lib.load()
    g = _lib.Grid()
    g.dim = dim
    for d in range(3):
        g.n[d] = int(n[d]) if d < dim else 1
    o = _options(precision=precision, solver=solver)
    out = ctypes.c_size_t()
    _check(L.pt_problem_estimate_bytes(ctypes.byref(g), int(N), ctypes.byref(o), ctypes.byref(out)))
    return int(out.value)


class Server:
    """Continuous-batching solve server on the current device (wraps ``pt_server``)."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 0):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        _check(self._lib.pt_server_create(int(hbm_budget), int(max_active), ctypes.byref(h)))
        self._h = h

    def submit(self, dim, n, N, T, coeff, f=None, seed: int = 0, u0=None, tol: float = 1e-8,
               max_it: int = 2000, taus=None, **opts) -> int:
        g = _lib.Grid()
        g.dim = dim
        for d in range(3):
            g.n[d] = int(n[d]) if d < dim else 1
        fp, fdev = _ptr(f)
        up, udev = _ptr(u0)
        if fdev or udev:
            raise ValueError("server requests take host arrays")
        steps = _step_array(taus, int(N))
        o = _options(steps=steps, **opts)
        t = ctypes.c_ulonglong()
        _check(self._lib.pt_server_submit(self._h, ctypes.byref(g), int(N), float(T), ctypes.byref(_coeff(coeff)),
                                          fp, int(seed) & 0xFFFFFFFFFFFFFFFF, up, ctypes.byref(o), float(tol),
                                          int(max_it), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, u_out=None, timeout_ms: int = -1):
        """Returns (solve status, iterations); raises PtError (e.g. PT_ETIMEOUT)."""
        up, _ = _ptr(u_out)
        it, stt = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.pt_server_wait(self._h, ctypes.c_ulonglong(ticket), int(timeout_ms), up,
                                        ctypes.byref(it), ctypes.byref(stt)))
        return stt.value, it.value

    def stats(self):
        p50, p99, rate = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        done = ctypes.c_int()
        _check(self._lib.pt_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(rate),
                                         ctypes.byref(done)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "dofs_per_s": rate.value, "completed": done.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pt_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batch(problems, tol, max_it):
    """Solve several problems together (pt_solve_batch); returns (iters, statuses) lists.
    ``tol`` and ``max_it`` are scalars or per-problem sequences."""
    count = len(problems)
    tols = [float(tol)] * count if np.isscalar(tol) else [float(t) for t in tol]
    mits = [int(max_it)] * count if np.isscalar(max_it) else [int(m) for m in max_it]
    hs = (ctypes.c_void_p * count)(*[p.handle.value for p in problems])
    t = (ctypes.c_double * count)(*tols)
    m = (ctypes.c_int * count)(*mits)
    it = (ctypes.c_int * count)()
    stt = (ctypes.c_int * count)()
    _check(_lib.load().pt_solve_batch(hs, count, t, m, it, stt))
    return list(it), list(stt)


def dst_forward_noalloc(r, out, stream: Optional[int] = None):
    """Forward temporal transform of the columns of ``r`` ([N_t][ncols] float64 CUDA tensor)
    into ``out`` without any device allocation by the library (``pt_dst_forward_noalloc``).
    For callers whose device memory belongs to another allocator; calls that overlap on the
    GPU share one scratch array and must not run concurrently."""
    rp, rdev = _ptr(r)
    op, odev = _ptr(out)
    if not (rdev and odev):
        raise ValueError("dst_forward_noalloc takes device tensors")
    N, ncols = int(r.shape[0]), int(r.numel() // r.shape[0])
    _check(_lib.load().pt_dst_forward_noalloc(rp, op, N, ncols, stream))
    return out


def _ptr(a) -> tuple:
    """(address, on_device) of a NumPy array or a torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    # torch tensor
    if str(a.dtype) != "torch.float64" or not a.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return a.data_ptr(), (1 if a.is_cuda else 0)


def _coeff(c) -> _lib.Coeff:
    k = _lib.Coeff()
    k.a0 = float(c.a0)
    k.c = float(c.c)
    for d in range(3):
        k.fx[d] = int(c.fx[d])
        k.mx[d] = float(c.mx[d])
    k.ft = int(c.ft)
    k.mt = float(c.mt)
    return k


class Problem:
    """One time-global problem resident on the GPU (wraps ``pt_problem``).

    ``coeff`` is any object with attributes a0, c, fx[3], mx[3], ft, mt (see ``pt_coeff``).
    ``f``: [N][n_s] source values, NumPy (host) or torch CUDA tensor (device), float64.
    ``taus``: the N step lengths tau_1..tau_N (summing to T), or None for uniform steps T/N.
    ``mass``: "identity" (finite differences, M = I) or "p1" (P1 finite elements, ``pt_options.mass``).
    """

    def __init__(self, dim: int, n: Sequence[int], N: int, T: float, coeff, f, u0=None,
                 precision: str = "fp64", omega: float = 0.0, solver: str = "mg",
                 stream: Optional[int] = None, check_every: int = 0, jacobi_weight: float = 0.0,
                 autotune=0, dst_cols: int = 0, coarse_elems: int = 0,
                 graphs: bool = True, n_vcycles: int = 0, h_solver: str = "auto", krylov: int = 0,
                 taus=None, mass: str = "identity"):
        L = _lib.load()
        self._lib = L
        self.dim, self.n, self.N, self.T = dim, list(n)[:dim], N, float(T)
        self.ns = int(np.prod(self.n))
        g = _lib.Grid()
        g.dim = dim
        for d in range(3):
            g.n[d] = int(n[d]) if d < dim else 1
        opts = _lib.Options()
        opts.precision = {"fp64": _lib.PT_PREC_FP64, "mixed": _lib.PT_PREC_MIXED}[precision]
        opts.omega = float(omega)
        opts.spatial_solver = {"mg": _lib.PT_SOLVER_MG, "exact": _lib.PT_SOLVER_EXACT_1D}[solver]
        opts.n_vcycles = int(n_vcycles)
        opts.jacobi_weight = float(jacobi_weight)
        opts.stream = stream
        opts.check_every = int(check_every)
        opts.autotune = 1 if autotune is True else (-1 if autotune is False else int(autotune))
        opts.dst_cols = int(dst_cols)
        opts.coarse_elems = int(coarse_elems)
        opts.no_graphs = 0 if graphs else 1
        opts.h_solver = {"auto": 0, "vcycle": 1, "exact": 2}[h_solver]
        opts.krylov = int(krylov)
        opts.mass = {"identity": 0, "p1": 1}[mass]
        steps = _step_array(taus, int(N))
        if steps is not None:
            opts.tau_steps = steps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._opts = opts
        self._steps = steps  # tau_steps points into it
        fp, fdev = _ptr(f)
        up, udev = _ptr(u0)
        h = ctypes.c_void_p()
        _check(L.pt_problem_create(ctypes.byref(g), int(N), float(T), ctypes.byref(_coeff(coeff)),
                                   fp, fdev, up, udev, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def set_rhs(self, f, u0=None):
        fp, fdev = _ptr(f)
        up, udev = _ptr(u0)
        _check(self._lib.pt_problem_set_rhs(self._h, fp, fdev, up, udev))

    def set_rhs_uniform(self, seed: int, u0=None):
        """Source f = U(-1,1) per space-time node from SplitMix64(seed), generated on the device."""
        up, udev = _ptr(u0)
        _check(self._lib.pt_problem_set_rhs_uniform(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, up, udev))

    def solve(self, tol: float, max_it: int, u_out=None, with_history: bool = True):
        """Run the Uzawa iteration; returns (status, iters, history).

        ``u_out`` (NumPy or torch, [N][n_s] float64) receives the solution if given.
        ``status`` is PT_OK, PT_ENOTCONV or PT_EDIVERGED (other statuses raise)."""
        up, udev = _ptr(u_out)
        hist = np.zeros(max_it + 1) if with_history else None
        it = ctypes.c_int(0)
        hp = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if hist is not None else None
        st = _check(self._lib.pt_solve(self._h, float(tol), int(max_it), up, udev, hp, ctypes.byref(it)),
                    allowed=(PT_OK, PT_ENOTCONV, PT_EDIVERGED))
        return st, it.value, (hist[: it.value + 1] if hist is not None else None)

    def device_bytes(self) -> int:
        """Device memory this problem holds."""
        out = ctypes.c_size_t()
        _check(self._lib.pt_problem_device_bytes(self._h, ctypes.byref(out)))
        return int(out.value)

    def get_state(self, u_out=None, p_out=None):
        """Copy the current iterates (u_j, p_j) into the given arrays (both host or both device)."""
        up, udev = _ptr(u_out)
        pp, pdev = _ptr(p_out)
        if u_out is not None and p_out is not None and udev != pdev:
            raise ValueError("u_out and p_out must both be host or both be device arrays")
        _check(self._lib.pt_problem_get_state(self._h, up, pp, udev or pdev))
        return u_out, p_out

    def _component(self, name: str, x, out):
        xp, xdev = _ptr(x)
        op, odev = _ptr(out)
        if not (xdev and odev):
            raise ValueError("component calls take device tensors")
        _check(getattr(self._lib, name)(self._h, xp, op))
        return out

    def apply_B(self, u, out):
        return self._component("pt_apply_B", u, out)

    def apply_S(self, u, out):
        """out = S u, the Schur complement of eq. 2.5 with the problem's A~ (FP64 problems)."""
        return self._component("pt_apply_S", u, out)

    def dst_forward(self, r, out):
        return self._component("pt_dst_forward", r, out)

    def dst_inverse(self, y, out):
        return self._component("pt_dst_inverse", y, out)

    def precond_A(self, r, out):
        return self._component("pt_precond_A", r, out)

    def precond_H(self, r, out):
        return self._component("pt_precond_H", r, out)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pt_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
