"""Host-side checks of the C ABI that need no GPU: the library loads, exports every entry
point declared in include/pt.h, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1802_08126_gb300 as ptu
from paper_1802_08126_gb300 import _lib, build
import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pt_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for n in _lib.EXPORTED:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _create(lib, dim=2, n=7, N=8, c=0.5, a0=1.0, solver=0, nv=0, mass=0, krylov=0, precision=0, steps=None,
            h_solver=0):
    g = _lib.Grid()
    g.dim = dim
    for d in range(3):
        g.n[d] = n
    k = _lib.Coeff()
    k.a0, k.c = a0, c
    o = _lib.Options()
    o.spatial_solver = solver
    o.n_vcycles = nv
    o.mass = mass
    o.h_solver = h_solver
    o.krylov = krylov
    o.precision = precision
    if steps is not None:
        steps = np.ascontiguousarray(steps, dtype=np.float64)
        o.tau_steps = steps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    f = np.zeros(N * n ** dim)
    h = ctypes.c_void_p()
    st = lib.pt_problem_create(ctypes.byref(g), N, 1.0, ctypes.byref(k), f.ctypes.data, 0, None, 0,
                               ctypes.byref(o), ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw", [dict(n=6), dict(N=3000), dict(N=0), dict(dim=4), dict(c=1.0),
                                dict(solver=1, dim=2), dict(nv=5), dict(mass=2), dict(mass=-1), dict(krylov=65),
                                dict(mass=1, dim=3), dict(mass=1, precision=1), dict(mass=1, krylov=4),
                                dict(mass=1, h_solver=2),
                                dict(krylov=-1), dict(krylov=10, precision=1),
                                dict(steps=[0.125] * 7 + [0.0]), dict(steps=[0.125] * 7 + [-0.125]),
                                dict(steps=[0.125] * 7 + [float("nan")]), dict(steps=[0.125] * 7 + [0.126]),
                                dict(steps=[0.25] * 8)])
def test_invalid_arguments_rejected_on_host(lib, kw):
    st, h = _create(lib, **kw)
    assert st == _lib.PT_EINVAL
    assert h.value is None
    assert len(lib.pt_last_error()) > 0


def test_null_pointers_rejected(lib):
    assert lib.pt_solve(None, 1e-8, 10, None, 0, None, None) == _lib.PT_EINVAL
    assert lib.pt_apply_B(None, None, None) == _lib.PT_EINVAL
    assert lib.pt_apply_S(None, None, None) == _lib.PT_EINVAL
    lib.pt_problem_destroy(None)
    assert lib.pt_status_string(3) == b"PT_ENOTCONV"


def test_binding_rejects_wrong_dtype():
    with pytest.raises(ValueError):
        ptu._ptr(np.zeros(4, dtype=np.float32))


def test_memory_estimate_is_host_only_and_monotone():
    """pt_problem_estimate_bytes needs no device: it grows with N_t and the grid."""
    import paper_1802_08126_gb300 as ptu
    a = ptu.estimate_bytes(2, [255, 255], 64, "mixed")
    b = ptu.estimate_bytes(2, [255, 255], 128, "mixed")
    c = ptu.estimate_bytes(2, [511, 511], 64, "mixed")
    assert 0 < a < b and a < c
    assert ptu.estimate_bytes(3, [31, 31, 31], 16, "fp64") > 0
    assert ptu.estimate_bytes(1, [63], 64, "fp64", solver="exact") > 0
