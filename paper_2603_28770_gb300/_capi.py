"""ctypes declarations of the C ABI in include/zeus.h.

Argument marshalling only: every step of the method runs in the CUDA
kernels of libzeus.so.  Loading fails loudly if the library cannot be built
or loaded; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

ZEUS_OK = 0
ZEUS_EINVAL = -1
ZEUS_ENOMEM = -2
ZEUS_ECUDA = -3
ZEUS_ETIMEOUT = -4
ZEUS_EUNSUPPORTED = -5
ZEUS_EWORKSPACE = -6

OBJECTIVES = {"rosenbrock": 0, "rastrigin": 1, "ackley": 2, "goldstein_price": 3, "quadratic": 100}
OBJ_USER = 200  # objective id of user objective k: OBJ_USER + k (include/zeus_user.cuh)
PRECISIONS = {"fp64": 0, "fp32_guarded": 1}
GRAD_MODES = {"forward": 0, "adjoint": 1}
RUN_STATUS = {0: "max_iter", 1: "converged", 2: "stopped", 3: "nonfinite", 4: "stalled"}


class zeus_problem(C.Structure):
    _fields_ = [
        ("objective", C.c_int32), ("dim", C.c_int32),
        ("lower", C.c_double), ("upper", C.c_double),
        ("n_starts", C.c_int64),
        ("pso_iters", C.c_int32), ("bfgs_max_iters", C.c_int32),
        ("ls_max_iters", C.c_int32), ("required_converged", C.c_int32),
        ("grad_tol", C.c_double),
        ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
        ("armijo_c", C.c_double), ("backtrack", C.c_double),
        ("target_f", C.c_double),
        ("seed", C.c_uint64),
        ("precision", C.c_int32), ("grad_mode", C.c_int32),
        ("start_from_pbest", C.c_int32), ("threads_per_start", C.c_int32),
        ("lbfgs_m", C.c_int32), ("pad", C.c_int32),
    ]


class zeus_result(C.Structure):
    _fields_ = [
        ("best_f", C.c_double), ("best_index", C.c_int64),
        ("n_converged", C.c_int64), ("total_iters", C.c_int64),
        ("total_feval", C.c_int64), ("gbest_f", C.c_double),
        ("gbest_index", C.c_int64), ("error", C.c_int32), ("stop_flag", C.c_int32),
        ("h_reads", C.c_int64), ("h_writes", C.c_int64),
    ]


class zeus_plan(C.Structure):
    _fields_ = [("narrow", C.c_int32), ("handover", C.c_int32), ("block", C.c_int32),
                ("stream", C.c_int32), ("blocks", C.c_int32), ("lbfgs", C.c_int32),
                ("warp", C.c_int32), ("h_bytes", C.c_int64)]


BATCH_MAX_CLASSES = 32


class zeus_batch_plan(C.Structure):
    _fields_ = [("n_problems", C.c_int32), ("pso_blocks", C.c_int32), ("items", C.c_int32),
                ("pso_iters_max", C.c_int32), ("q_cap", C.c_int32), ("d_max_handover", C.c_int32),
                ("precision", C.c_int32), ("grad_mode", C.c_int32), ("n_classes", C.c_int32),
                ("handover_smem", C.c_int32), ("n_user", C.c_int32), ("pad", C.c_int32),
                ("class_first", C.c_int32 * BATCH_MAX_CLASSES),
                ("class_count", C.c_int32 * BATCH_MAX_CLASSES),
                ("class_smem", C.c_int32 * BATCH_MAX_CLASSES),
                ("class_kind", C.c_int32 * BATCH_MAX_CLASSES),
                ("total_starts", C.c_int64), ("total_coords", C.c_int64), ("total_g", C.c_int64),
                ("workspace_bytes", C.c_uint64), ("table_bytes", C.c_uint64)]


CLUSTER_METHODS = {"f": 0, "x": 1}
CLUSTER_MAX = 4096
LABEL_NONE, LABEL_LEFT = -1, -2


class zeus_cluster_params(C.Structure):
    _fields_ = [("method", C.c_int32), ("max_clusters", C.c_int32), ("only_converged", C.c_int32),
                ("pad", C.c_int32), ("tol", C.c_double)]


class zeus_cluster_result(C.Structure):
    _fields_ = [("n_candidates", C.c_int64), ("n_clusters", C.c_int64), ("n_left", C.c_int64),
                ("best_count", C.c_int64), ("best_leader", C.c_int64), ("best_f", C.c_double),
                ("best_spread", C.c_double), ("error", C.c_int32), ("pad", C.c_int32)]


class ZeusError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


_VP = C.c_void_p
_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); exactly the declarations of include/zeus.h
SIGNATURES = {
    "zeus_strerror": (C.c_char_p, [C.c_int]),
    "zeus_abi_version": (C.c_int, []),
    "zeus_set_wait_limit": (C.c_int, [C.c_uint32]),
    "zeus_default_problem": (C.c_int, [C.POINTER(zeus_problem)]),
    "zeus_validate": (C.c_int, [C.POINTER(zeus_problem)]),
    "zeus_workspace_size": (C.c_int, [C.POINTER(zeus_problem), C.POINTER(C.c_size_t)]),
    "zeus_plan_info": (C.c_int, [C.POINTER(zeus_problem), C.POINTER(zeus_plan)]),
    "zeus_solve": (C.c_int, [C.POINTER(zeus_problem), _VP, C.c_size_t, _VP, _VP, _VP, _VP, _VP,
                             _VP, _VP]),
    "zeus_solve_from": (C.c_int, [C.POINTER(zeus_problem), _VP, _VP, C.c_size_t, _VP, _VP, _VP,
                                  _VP, _VP, _VP, _VP]),
    "zeus_pso": (C.c_int, [C.POINTER(zeus_problem), _VP, C.c_size_t, _VP, _VP, _VP, _VP, _VP,
                           _VP, _VP]),
    "zeus_objective_eval": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _VP, _VP, _VP, C.c_int32,
                                      _VP]),
    "zeus_objective_eval_f32": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _VP, _VP, _VP,
                                          C.c_int32, _VP]),
    "zeus_argmin": (C.c_int, [_VP, C.c_int64, _VP, C.c_size_t, _VP, _VP]),
    "zeus_argmin_workspace_size": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "zeus_uniform": (C.c_int, [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, C.c_int32, _VP,
                               _VP]),
    "zeus_math_eval": (C.c_int, [C.c_int32, C.c_int64, _VP, _VP, _VP, _VP]),
    "zeus_cluster_workspace_size": (C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
    "zeus_cluster": (C.c_int, [C.POINTER(zeus_cluster_params), C.c_int64, C.c_int32, _VP, _VP, _VP,
                               _VP, _VP, _VP, _VP, _VP, C.c_size_t, _VP]),
    "zeus_batch_cluster": (C.c_int, [C.POINTER(zeus_batch_plan), _VP, C.c_size_t,
                                     C.POINTER(zeus_cluster_params), _VP, _VP, _VP, _VP, _VP, _VP,
                                     _VP, _VP]),
    "zeus_user_objective_count": (C.c_int32, []),
    "zeus_user_objective_info": (C.c_int, [C.c_int32, C.c_char_p, C.c_int32,
                                           C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "zeus_batch_plan_make": (C.c_int, [C.POINTER(zeus_problem), C.c_int32,
                                       C.POINTER(zeus_batch_plan)]),
    "zeus_batch_prepare": (C.c_int, [C.POINTER(zeus_problem), C.c_int32,
                                     C.POINTER(zeus_batch_plan), _VP, C.c_size_t, _VP]),
    "zeus_batch_solve": (C.c_int, [C.POINTER(zeus_batch_plan), _VP, C.c_size_t, _VP, _VP, _VP,
                                   _VP, _VP, _VP, _VP]),
    "zeus_solve_from_noalloc": (C.c_int, [C.POINTER(zeus_problem), _VP, _VP, _VP, _VP, _VP,
                                          _VP, _VP, _VP]),
    "zeus_context_create": (C.c_int, [C.POINTER(_VP)]),
    "zeus_context_destroy": (C.c_int, [_VP]),
    "zeus_solve_host": (C.c_int, [_VP, C.POINTER(zeus_problem), _VP, _VP, _VP, _VP, _VP, _VP,
                                  _VP]),
}


def library_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load libzeus.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libzeus.so missing at {path}")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            if L.zeus_abi_version() != 2:
                raise RuntimeError("libzeus.so ABI version mismatch")
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().zeus_strerror(int(code)).decode()


def check(code: int, where: str) -> None:
    if code != ZEUS_OK:
        raise ZeusError(code, where)


def user_objectives() -> dict:
    """The user objectives compiled into libzeus.so (its plug-in header):
    name -> (objective id, min_dim, max_dim); max_dim 0 = no limit."""
    L = lib()
    out = {}
    buf = C.create_string_buffer(64)
    lo, hi = C.c_int32(), C.c_int32()
    for k in range(L.zeus_user_objective_count()):
        check(L.zeus_user_objective_info(k, buf, 64, C.byref(lo), C.byref(hi)),
              "zeus_user_objective_info")
        out[buf.value.decode()] = (OBJ_USER + k, lo.value, hi.value)
    return out


def objective_code(o) -> int:
    """Objective id of a built-in or user objective name (ids pass through)."""
    if not isinstance(o, str):
        return int(o)
    if o in OBJECTIVES:
        return OBJECTIVES[o]
    user = user_objectives()
    if o in user:
        return user[o][0]
    raise KeyError(f"unknown objective {o!r}: built in {sorted(OBJECTIVES)}, user {sorted(user)}")
