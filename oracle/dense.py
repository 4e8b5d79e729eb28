"""O1: the plain FP64 definition of the IMQ product (TEST INFRASTRUCTURE ONLY).

Paper Section 2: Eq. (4) A c = f with a_ij = phi(|x_i - y_j|), Eq. (5)
phi(r) = 1/sqrt(t^2 + r^2) (t is the shape parameter, called c here), and the
interpolant Eq. (2).  The loops live in ``dense.c`` (plain C, FP64, OpenMP over
rows, sequential j); this module builds it with gcc on first use and wraps it
with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_dense.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dense.c with gcc (-O2, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "dense.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.oracle_dense_matvec.argtypes = [P, I64, D, P, P, ctypes.c_int]
            lib.oracle_dense_rows.argtypes = [P, I64, D, P, P, I64, P]
            lib.oracle_evaluate.argtypes = [P, I64, P, I64, D, P, P, ctypes.c_int]
            lib.oracle_evaluate_transpose.argtypes = [P, I64, P, I64, D, P, P]
            lib.oracle_assemble.argtypes = [P, I64, D, P, ctypes.c_int]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def matvec(points, c: float, u) -> np.ndarray:
    """b = A u, FP64, u of shape (n,) or (nrhs, n)."""
    pts = _c(points)
    u = _c(u)
    n = pts.shape[0]
    nrhs = 1 if u.ndim == 1 else u.shape[0]
    b = np.empty_like(u)
    if n:
        _load().oracle_dense_matvec(_ptr(pts), n, float(c), _ptr(u), _ptr(b), nrhs)
    return b


def matvec_rows(points, c: float, u, rows) -> np.ndarray:
    """(A u)_i for i in rows, exact FP64 (used for sampled checks at large N)."""
    pts = _c(points)
    u = _c(u)
    rows = _c(rows, np.int64)
    b = np.empty(rows.shape[0])
    _load().oracle_dense_rows(_ptr(pts), pts.shape[0], float(c), _ptr(u), _ptr(rows),
                              rows.shape[0], _ptr(b))
    return b


def evaluate(src, c: float, coef, targets, deriv: bool = False) -> np.ndarray:
    """P(t_k) = sum_j coef_j phi(|t_k - x_j|) (Eq. (2)); deriv -> d phi / dc kernel."""
    s, t, w = _c(src), _c(targets), _c(coef)
    out = np.empty(t.shape[0])
    _load().oracle_evaluate(_ptr(s), s.shape[0], _ptr(t), t.shape[0], float(c), _ptr(w),
                            _ptr(out), 1 if deriv else 0)
    return out


def evaluate_transpose(src, c: float, r, targets) -> np.ndarray:
    """E^T r with E_kj = phi(|t_k - x_j|)."""
    s, t, r = _c(src), _c(targets), _c(r)
    out = np.empty(s.shape[0])
    _load().oracle_evaluate_transpose(_ptr(s), s.shape[0], _ptr(t), t.shape[0], float(c),
                                      _ptr(r), _ptr(out))
    return out


def assemble(points, c: float, deriv: bool = False) -> np.ndarray:
    """The dense matrix A (or dA/dc), small N only."""
    pts = _c(points)
    n = pts.shape[0]
    A = np.empty((n, n))
    _load().oracle_assemble(_ptr(pts), n, float(c), _ptr(A), 1 if deriv else 0)
    return A


def matvec_dc(points, c: float, u) -> np.ndarray:
    """(dA/dc) u with dA/dc = -c (r^2+c^2)^{-3/2}."""
    pts = _c(points)
    return evaluate(pts, c, u, pts, deriv=True)
