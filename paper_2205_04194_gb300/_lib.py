"""ctypes binding of libimq.so (include/imq.h): symbol signatures and status checks.

Argument marshalling only; every computation runs in the CUDA library.  There
is no fallback: if the shared library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double
INT = ctypes.c_int
CHAR = ctypes.c_char


class ImqError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func}: {status_name(status)}: {msg}")


# caller-supplied allocator of a plan's device buffers (imq_options.alloc / free)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class ImqOptions(ctypes.Structure):
    _fields_ = [("struct_size", I32), ("has_domain", I32), ("x0", D), ("y0", D), ("side", D),
                ("check_duplicates", I32), ("m2l_kernel", I32), ("algorithm", I32), ("levels", I32),
                ("translations", I32), ("p2p_warps", I32), ("p2p_chunk", I32), ("m2l_stages", I32),
                ("m2l_split", I32), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", P)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_points", I64), ("n_nodes", I64), ("n_problems", I32), ("algorithm", I32), ("n_boxes", I32), ("n_leaves", I32), ("max_level", I32), ("p", I32),
                ("leaf", I32), ("k_real", I32), ("x0", D), ("y0", D), ("side", D), ("c", D),
                ("n_u", I64), ("n_v", I64), ("n_w", I64), ("n_x", I64), ("p2p_pairs", I64),
                ("m2l_pairs", I64), ("device_bytes", I64)]


class CgOptions(ctypes.Structure):
    _fields_ = [("struct_size", I32), ("rtol", D), ("maxit", I32), ("precond", I32), ("schwarz_nmax", I32),
                ("schwarz_shift", D), ("refine_steps", I32), ("inner_rtol", D), ("residual", I32),
                ("x0_given", I32), ("residual_plan", P), ("inner_operator", I32), ("schwarz_fp64", I32),
                ("coarse_points", I32), ("coarse_gram", I32), ("krylov", I32), ("gmres_m", I32),
                ("reserved", I32 * 2)]


class CgInfo(ctypes.Structure):
    _fields_ = [("iterations", I32), ("outer_steps", I32), ("status", INT), ("max_rel_residual", D),
                ("seconds", D), ("rel_residual", D * 16)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("p", I32), ("leaf", I32), ("rel_err", D), ("matvec_ms", ctypes.c_float),
                ("translations", I32), ("p2p_warps", I32), ("p2p_chunk", I32), ("m2l_stages", I32),
                ("m2l_split", I32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("p", I32), ("leaf", I32), ("rel_err", D), ("matvec_ms", ctypes.c_float), ("met", I32),
                ("n_tried", I32), ("sampled_rows", I32), ("translations", I32), ("p2p_warps", I32),
                ("p2p_chunk", I32), ("m2l_stages", I32), ("m2l_split", I32), ("reserved", I32),
                ("tried", TuneEntry * 64)]


# name -> (restype, argtypes)
SIGNATURES = {
    "imq_plan": (INT, [P, I64, D, INT, INT, P, P, P]),
    "imq_plan_eval": (INT, [P, I64, P, I64, D, INT, INT, P, P, P]),
    "imq_plan_batched": (INT, [P, P, INT, P, INT, INT, P, P, P]),
    "imq_plan_destroy": (None, [P]),
    "imq_matvec_dc": (INT, [P, P, P, INT, INT, P]),
    "imq_evaluate": (INT, [P, P, P, INT, INT, P]),
    "imq_evaluate_transpose": (INT, [P, P, P, INT, INT, P]),
    "imq_evaluate_dc": (INT, [P, P, P, INT, INT, P]),
    "imq_matvec": (INT, [P, P, P, INT, INT, P]),
    "imq_matvec_timed": (INT, [P, P, P, INT, INT, P, P, INT, P]),
    "imq_dense_matvec": (INT, [P, I64, D, P, P, INT, INT, P]),
    "imq_cg_default_options": (None, [P]),
    "imq_cg_solve": (INT, [P, P, P, INT, P, P, P]),
    "imq_cg_solve_batched": (INT, [P, P, P, INT, P, P, P, P, P]),
    "imq_interp_loss_grad": (INT, [P, P, P, P, P, INT, P, P, P, P, P, P]),
    "imq_dense_matvec_noalloc": (INT, [P, I64, D, P, P, P]),
    "imq_autotune": (INT, [P, P, INT, P, D, P, INT, P, INT, INT, P, P, P]),
    "imq_autotune_v": (INT, [P, P, INT, P, D, P, INT, P, INT, INT, P, P, P, P]),
    "imq_sync_check": (INT, [P]),
    "imq_selftest_wait_timeout": (INT, [P]),
    "imq_plan_get_info": (INT, [P, P]),
    "imq_plan_export_tree": (INT, [P, P, P, P, P, P, P, P, P]),
    "imq_plan_export_list": (INT, [P, CHAR, P, P]),
    "imq_status_string": (ctypes.c_char_p, [INT]),
    "imq_last_error": (ctypes.c_char_p, []),
    "imq_version": (ctypes.c_char_p, []),
}


def load(path: str | None = None):
    """Load libimq.so (built by ``paper_2205_04194_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or LIB
            if not os.path.exists(so):
                raise RuntimeError(f"libimq.so not built ({so}); run paper_2205_04194_gb300.build.build()")
            lib = ctypes.CDLL(so)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_name(status: int) -> str:
    try:
        return load().imq_status_string(int(status)).decode()
    except Exception:   # noqa: BLE001 - name lookup only
        return str(status)


def call(name: str, *args) -> int:
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise ImqError(st, name, lib.imq_last_error().decode())
    return st
