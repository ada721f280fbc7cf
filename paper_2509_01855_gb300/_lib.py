"""ctypes binding of libbirkhoff.so: argument marshalling only.

Every operation runs in the CUDA library; this module turns torch tensors into device pointers
and sizes and checks the returned status. If the shared library is missing the import fails
with an error: there is no fallback path.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbirkhoff.so")

BK_F64, BK_F32 = 0, 1
BK_DBL_INT, BK_ORBIT, BK_BILINEAR, BK_ORBIT_MT = 0, 1, 2, 3
BK_OP_STATE, BK_OP_KKT = 0, 1
BK_BARRIER_PRIMAL, BK_BARRIER_PRIMAL_DUAL = 0, 1
STATUS = {0: "BK_OK", 1: "BK_ERR_ARG", 2: "BK_ERR_CUDA", 3: "BK_ERR_OOM",
          4: "BK_ERR_NOT_CONVERGED", 5: "BK_ERR_TIMEOUT", 6: "BK_ERR_INFEASIBLE",
          7: "BK_ERR_UNSUPPORTED"}

# Symbols declared in include/birkhoff.h (checked by the CPU test suite).
EXPORTS = ["bk_last_error", "bk_version", "bk_launch_count", "bk_plan_create", "bk_plan_destroy", "bk_plan_info",
           "bk_plan_grid", "birkhoff_apply", "birkhoff_apply_T", "birkhoff_apply_noalloc", "bk_plan_set_dense",
           "bk_plan_dense_state", "bk_plan_dense_check", "bk_plan_shape", "bk_set_f64_transform", "bk_plan_f64_mode",
           "bk_plan_dense_test_timeout", "birkhoff_apply_b", "birkhoff_apply_b_T",
           "bk_set_f64_precond", "bk_problem_precond_dtype", "bk_set_krylov_graphs", "bk_set_krylov_wait_limit", "birkhoff_apply_batch",
           "bk_problem_create",
           "bk_problem_destroy", "bk_problem_set_params", "bk_problem_set_control_bounds", "bk_problem_set_terminal_bounds", "bk_problem_set_barrier", "bk_problem_device_bytes", "bk_problem_info", "bk_linearize", "kkt_apply",
           "precond_apply", "bk_krylov_workspace_bytes", "krylov_solve",
           "bk_newton_workspace_bytes", "newton_solve", "bk_kkt_residual", "bk_min_time_seed",
           "bk_abi_struct_size"]


class BirkhoffError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class KrylovOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("use_precond", ctypes.c_int)]


class KrylovInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("converged", ctypes.c_int)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("krylov_rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_krylov", ctypes.c_int), ("ir_rtol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("precond_reuse", ctypes.c_int),
                ("weighted_inner", ctypes.c_int)]


class NewtonInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("krylov_iterations", ctypes.c_int),
                ("kkt_solves", ctypes.c_int), ("backtracks", ctypes.c_int),
                ("residual", ctypes.c_double), ("residual0", ctypes.c_double),
                ("converged", ctypes.c_int), ("precond_builds", ctypes.c_int)]


_lib = None


def lib():
    """Load libbirkhoff.so once; raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbirkhoff.so not built (run paper_2509_01855_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "bk_last_error": (ctypes.c_char_p, []),
        "bk_version": (ctypes.c_char_p, []),
        "bk_launch_count": (ctypes.c_uint64, []),
        "bk_plan_create": (c_int, [ctypes.POINTER(vp), i64, c_int, c_int, c_int, dbl, dbl, i64, vp]),
        "bk_plan_destroy": (None, [vp]),
        "bk_plan_info": (c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                 ctypes.POINTER(c_int)]),
        "bk_plan_grid": (c_int, [vp, vp, vp]),
        "birkhoff_apply": (c_int, [vp, vp, vp, c_int, vp]),
        "birkhoff_apply_T": (c_int, [vp, vp, vp, c_int, vp]),
        "birkhoff_apply_noalloc": (c_int, [vp, vp, i64, c_int, i64, dbl, dbl, vp]),
        "bk_plan_set_dense": (c_int, [vp, c_int, vp]),
        "bk_plan_dense_check": (c_int, [vp, ctypes.POINTER(c_int)]),
        "bk_plan_dense_state": (c_int, [vp, ctypes.POINTER(c_int)]),
        "bk_set_f64_transform": (c_int, [c_int]),
        "bk_plan_f64_mode": (c_int, [vp, ctypes.POINTER(c_int)]),
        "bk_plan_dense_test_timeout": (c_int, [vp, c_int]),
        "birkhoff_apply_b": (c_int, [vp, vp, vp, c_int, vp]),
        "birkhoff_apply_b_T": (c_int, [vp, vp, vp, c_int, vp]),
        "bk_set_f64_precond": (c_int, [c_int]),
        "bk_set_krylov_graphs": (c_int, [c_int]),
        "birkhoff_apply_batch": (c_int, [vp, vp, vp, vp, c_int, c_int, vp]),
        "bk_set_krylov_wait_limit": (c_int, [ctypes.c_double]),
        "bk_problem_precond_dtype": (c_int, [vp, ctypes.POINTER(c_int)]),
        "bk_plan_shape": (c_int, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                  ctypes.POINTER(c_int)]),
        "bk_problem_create": (c_int, [ctypes.POINTER(vp), c_int, ctypes.POINTER(dbl), c_int, i64,
                                      c_int, dbl, dbl, vp]),
        "bk_problem_destroy": (None, [vp]),
        "bk_problem_set_params": (c_int, [vp, ctypes.POINTER(dbl), c_int, dbl, dbl]),
        "bk_problem_set_control_bounds": (c_int, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), c_int]),
        "bk_problem_set_terminal_bounds": (c_int, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), c_int]),
        "bk_problem_set_barrier": (c_int, [vp, dbl, dbl, c_int]),
        "bk_problem_device_bytes": (ctypes.c_size_t, [vp]),
        "bk_problem_info": (c_int, [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                    ctypes.POINTER(c_int), ctypes.POINTER(i64),
                                    ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "bk_linearize": (c_int, [vp, vp, vp]),
        "kkt_apply": (c_int, [vp, c_int, vp, vp, vp]),
        "precond_apply": (c_int, [vp, c_int, vp, vp, c_int, vp]),
        "bk_krylov_workspace_bytes": (ctypes.c_size_t, [vp, c_int, c_int]),
        "krylov_solve": (c_int, [vp, c_int, vp, vp, ctypes.POINTER(KrylovOpts),
                                 ctypes.POINTER(KrylovInfo), vp, vp]),
        "bk_newton_workspace_bytes": (ctypes.c_size_t, [vp, c_int]),
        "newton_solve": (c_int, [vp, vp, ctypes.POINTER(NewtonOpts), ctypes.POINTER(NewtonInfo),
                                 vp, vp]),
        "bk_kkt_residual": (c_int, [vp, vp, vp, ctypes.POINTER(dbl), vp]),
        "bk_min_time_seed": (c_int, [vp, vp, vp, vp, vp]),
        "bk_abi_struct_size": (ctypes.c_size_t, [c_int]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    _lib = L
    return L


def check(status):
    if status != 0:
        raise BirkhoffError(status, lib().bk_last_error().decode())
    return status


def ptr(t):
    """Device (or host) address of a tensor, or None."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)
