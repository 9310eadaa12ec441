"""Build and ctypes binding of the C part of the oracle (``oracle.c``).

Test infrastructure only: see the package docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OcCoeff(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("c", ctypes.c_double),
                ("fx", ctypes.c_int * 3), ("mx", ctypes.c_double * 3),
                ("ft", ctypes.c_int), ("mt", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no fast-math) into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oc_implicit_euler.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.c_double,
                                            ctypes.POINTER(OcCoeff), dp, dp, dp, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int]
            L.oc_implicit_euler.restype = ctypes.c_int
            L.oc_apply_B.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(OcCoeff), dp, dp, ctypes.c_int, dp, ctypes.c_int]
            L.oc_apply_B.restype = None
            L.oc_apply_A.argtypes = [ctypes.c_int, ip, ctypes.c_double, ctypes.POINTER(OcCoeff),
                                     dp, dp, ctypes.c_int]
            L.oc_apply_A.restype = None
            L.oc_max_threads.argtypes = []
            L.oc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _coeff(k) -> OcCoeff:
    c = OcCoeff()
    c.a0 = float(k.a0)
    c.c = float(k.c)
    for d in range(3):
        c.fx[d] = int(k.fx[d])
        c.mx[d] = float(k.mx[d])
    c.ft = int(k.ft)
    c.mt = float(k.mt)
    return c


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iarr(n: Sequence[int]):
    arr = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    return arr


def _step_lengths(N: int, taus) -> Optional[np.ndarray]:
    if taus is None:
        return None
    taus = np.ascontiguousarray(taus, dtype=np.float64).reshape(-1)
    if taus.size != N:
        raise ValueError("need %d step lengths, got %d" % (N, taus.size))
    return taus


MASS = {"identity": 0, "p1": 1}


def implicit_euler(dim: int, n: Sequence[int], N: int, T: float, coeff, f: np.ndarray,
                   u0: Optional[np.ndarray] = None, steps: Optional[int] = None,
                   method: str = "cholesky", cg_tol: float = 1e-14, threads: int = 0,
                   taus: Optional[Sequence[float]] = None, mass: str = "identity") -> np.ndarray:
    """Sequential implicit Euler (§2, eq. 2.1) for steps 1..steps; returns [steps][ns].

    taus: the N step lengths tau_1..tau_N (t_n = tau_1 + ... + tau_n), or None for T/N.
    mass: "identity" (M = I, finite differences) or "p1" (the P1 mass matrix over h^d, dim <= 2;
    the source enters as the consistent load M f_n)."""
    steps = N if steps is None else steps
    tv = _step_lengths(N, taus)
    ns = int(np.prod(list(n)[:dim]))
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    if f.size < steps * ns:
        raise ValueError("f has %d values, need %d" % (f.size, steps * ns))
    u0c = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
    out = np.empty((steps, ns), dtype=np.float64)
    k = _coeff(coeff)
    rc = lib().oc_implicit_euler(dim, _iarr(n), N, float(T), ctypes.byref(k), _dptr(f), _dptr(u0c),
                                 _dptr(out), steps, 0 if method == "cholesky" else 1,
                                 float(cg_tol), int(threads), _dptr(tv), MASS[mass])
    if rc != 0:
        raise RuntimeError("oracle implicit Euler failed (code %d)" % rc)
    return out


def apply_B(dim: int, n: Sequence[int], N: int, T: float, coeff, u: np.ndarray,
            threads: int = 0, taus: Optional[Sequence[float]] = None, mass: str = "identity") -> np.ndarray:
    """B u = (K (x) M) u + diag(tau_n A_n) u, u_0 := 0 (§2, eq. 2.3-2.4); u is [N][ns]."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(N, -1)
    out = np.empty_like(u)
    k = _coeff(coeff)
    tv = _step_lengths(N, taus)
    lib().oc_apply_B(dim, _iarr(n), N, float(T), ctypes.byref(k), _dptr(u), _dptr(out), int(threads),
                     _dptr(tv), MASS[mass])
    return out


def apply_A(dim: int, n: Sequence[int], t: float, coeff, v: np.ndarray, threads: int = 0) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    out = np.empty_like(v)
    k = _coeff(coeff)
    lib().oc_apply_A(dim, _iarr(n), float(t), ctypes.byref(k), _dptr(v), _dptr(out), int(threads))
    return out


def max_threads() -> int:
    return int(lib().oc_max_threads())
