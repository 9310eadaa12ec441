"""ctypes declarations of the C ABI in ``include/pt.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libptuzawa.so")

PT_OK, PT_EINVAL, PT_ENOMEM, PT_ENOTCONV, PT_EDIVERGED, PT_ECUDA, PT_ETIMEOUT, PT_EBUSY = range(8)
PT_PREC_FP64, PT_PREC_MIXED = 0, 1
PT_SOLVER_MG, PT_SOLVER_EXACT_1D = 0, 1

EXPORTED = (
    "pt_problem_create", "pt_problem_set_rhs", "pt_solve", "pt_problem_destroy", "pt_last_error",
    "pt_status_string", "pt_apply_B", "pt_dst_forward", "pt_dst_inverse", "pt_precond_A",
    "pt_precond_H", "pt_kernel_launch_count", "pt_problem_get_state", "pt_profile_enable",
    "pt_profile_reset", "pt_profile_get", "pt_dst_forward_noalloc", "pt_solve_batch",
    "pt_problem_set_rhs_uniform", "pt_server_create", "pt_server_submit", "pt_server_wait",
    "pt_server_stats", "pt_server_destroy", "pt_problem_estimate_bytes", "pt_problem_device_bytes",
    "pt_apply_S",
)


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3)]


class Coeff(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("c", ctypes.c_double), ("fx", ctypes.c_int * 3),
                ("mx", ctypes.c_double * 3), ("ft", ctypes.c_int), ("mt", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("omega", ctypes.c_double),
                ("spatial_solver", ctypes.c_int), ("n_vcycles", ctypes.c_int),
                ("jacobi_weight", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("check_every", ctypes.c_int), ("autotune", ctypes.c_int), ("dst_cols", ctypes.c_int),
                ("coarse_elems", ctypes.c_int), ("no_graphs", ctypes.c_int), ("h_solver", ctypes.c_int),
                ("krylov", ctypes.c_int), ("mass", ctypes.c_int),
                ("tau_steps", ctypes.POINTER(ctypes.c_double))]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("CUDA solver library not built: %s is missing "
                               "(run paper_1802_08126_gb300.build.build())" % path)
        L = ctypes.CDLL(path)
        vp, dp, ip, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int
        L.pt_problem_create.argtypes = [ctypes.POINTER(Grid), i, ctypes.c_double, ctypes.POINTER(Coeff),
                                        vp, i, vp, i, ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.pt_problem_create.restype = i
        L.pt_problem_set_rhs.argtypes = [vp, vp, i, vp, i]
        L.pt_problem_set_rhs.restype = i
        L.pt_solve.argtypes = [vp, ctypes.c_double, i, vp, i, dp, ip]
        L.pt_solve.restype = i
        L.pt_problem_destroy.argtypes = [vp]
        L.pt_problem_destroy.restype = None
        L.pt_last_error.argtypes = []
        L.pt_last_error.restype = ctypes.c_char_p
        L.pt_status_string.argtypes = [i]
        L.pt_status_string.restype = ctypes.c_char_p
        for name in ("pt_apply_B", "pt_apply_S", "pt_dst_forward", "pt_dst_inverse", "pt_precond_A",
                     "pt_precond_H"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp]
            fn.restype = i
        L.pt_problem_get_state.argtypes = [vp, vp, vp, i]
        L.pt_problem_get_state.restype = i
        L.pt_problem_estimate_bytes.argtypes = [ctypes.POINTER(Grid), i, ctypes.POINTER(Options),
                                                ctypes.POINTER(ctypes.c_size_t)]
        L.pt_problem_estimate_bytes.restype = i
        L.pt_problem_device_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.pt_problem_device_bytes.restype = i
        L.pt_profile_enable.argtypes = [i]
        L.pt_profile_enable.restype = None
        L.pt_profile_reset.argtypes = []
        L.pt_profile_reset.restype = None
        L.pt_profile_get.argtypes = [i, ctypes.c_char_p, i, dp, dp, dp, ctypes.POINTER(ctypes.c_ulonglong)]
        L.pt_profile_get.restype = i
        L.pt_problem_set_rhs_uniform.argtypes = [vp, ctypes.c_ulonglong, vp, i]
        L.pt_problem_set_rhs_uniform.restype = i
        ull = ctypes.c_ulonglong
        L.pt_server_create.argtypes = [ctypes.c_size_t, i, ctypes.POINTER(vp)]
        L.pt_server_create.restype = i
        L.pt_server_submit.argtypes = [vp, ctypes.POINTER(Grid), i, ctypes.c_double, ctypes.POINTER(Coeff), vp,
                                       ull, vp, ctypes.POINTER(Options), ctypes.c_double, i, ctypes.POINTER(ull)]
        L.pt_server_submit.restype = i
        L.pt_server_wait.argtypes = [vp, ull, i, vp, ip, ip]
        L.pt_server_wait.restype = i
        L.pt_server_stats.argtypes = [vp, dp, dp, dp, ip]
        L.pt_server_stats.restype = i
        L.pt_server_destroy.argtypes = [vp]
        L.pt_server_destroy.restype = None
        L.pt_solve_batch.argtypes = [ctypes.POINTER(vp), i, dp, ip, ip, ip]
        L.pt_solve_batch.restype = i
        L.pt_dst_forward_noalloc.argtypes = [vp, vp, i, ctypes.c_longlong, vp]
        L.pt_dst_forward_noalloc.restype = i
        L.pt_kernel_launch_count.argtypes = []
        L.pt_kernel_launch_count.restype = ctypes.c_ulonglong
        _lib = L
        return _lib
