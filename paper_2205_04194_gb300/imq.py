"""Python surface of the IMQ library: the same entry points as include/imq.h.

Tensors are passed by pointer to the C ABI; CUDA tensors are used in place on
the current torch stream, host tensors / numpy arrays are copied by the
library inside the call.  Nothing here computes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CgInfo, CgOptions, ImqError, ImqOptions, PlanInfo, TuneResult, call

F32 = 0
F64 = 1


def _stream(stream=None) -> ctypes.c_void_p:
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _buf(a, dtype):
    """(pointer, keep-alive object) of a contiguous array of the given torch dtype."""
    if isinstance(a, torch.Tensor):
        if a.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    npdt = {torch.float64: np.float64, torch.float32: np.float32}[dtype]
    arr = np.ascontiguousarray(a, dtype=npdt)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _dtype_code(t) -> int:
    dt = t.dtype if isinstance(t, torch.Tensor) else np.asarray(t).dtype
    if dt in (torch.float32, np.float32):
        return F32
    if dt in (torch.float64, np.float64):
        return F64
    raise TypeError(f"unsupported dtype {dt}")


def _like(v, n_total: int, code: int):
    if isinstance(v, torch.Tensor):
        return torch.empty_like(v)
    return np.empty(np.shape(v), dtype=np.float32 if code == F32 else np.float64)


M2L_KERNELS = {"auto": 0, "cuda_cores": 1, "tensor": 2}


ALGORITHMS = {"fmm": 0, "treecode": 1}


def _torch_allocator():
    """(alloc, free) callbacks that serve a plan's device buffers from torch's caching
    allocator on the current device; keep them alive as long as the plan."""
    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:   # noqa: BLE001 - reported to the library as an allocation failure
            return None

    def _free(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return _lib.ALLOC_FN(_alloc), _lib.FREE_FN(_free)


TRANSLATIONS = {"fp32": 0, "fp64": 1, "mixed": 2}

# imq_cg_options fields by name (the values of include/imq.h's enums)
PRECONDS = {"none": 0, None: 0, "schwarz": 1, "schwarz2": 2}
RESIDUALS = {"plan": 0, "dense": 1}
OPERATORS = {"fast_f32": 0, "fast_f64": 1, "dense_f64": 2}
KRYLOVS = {"cg": 0, "gmres": 1}
COARSE_GRAMS = {"auto": 0, "fp64": 1, "fp32": 2}


def _plan_options(domain=None, check_duplicates=False, m2l_kernel="auto", algorithm="fmm", levels=0,
                  allocator=None, translations="fp32", p2p_warps=0, p2p_chunk=0, m2l_stages=0, m2l_split=0):
    opt = ImqOptions()
    opt.struct_size = ctypes.sizeof(ImqOptions)
    if allocator is not None:
        opt.alloc, opt.free = allocator
    if domain is not None:
        opt.has_domain = 1
        opt.x0, opt.y0, opt.side = (float(v) for v in domain)
    opt.check_duplicates = 1 if check_duplicates else 0
    opt.m2l_kernel = M2L_KERNELS[m2l_kernel]
    opt.algorithm = ALGORITHMS[algorithm]
    opt.levels = int(levels)
    opt.translations = TRANSLATIONS[translations]
    opt.p2p_warps, opt.p2p_chunk, opt.m2l_stages = int(p2p_warps), int(p2p_chunk), int(m2l_stages)
    opt.m2l_split = int(m2l_split)
    return opt


class Plan:
    """imq_plan: quadtree, interaction lists and operators for (points, c, p, leaf).

    algorithm="treecode" with levels=L builds the paper's Algorithm 1 on a uniform
    partition of 2^(L+1) x 2^(L+1) blocks at the finest level (leaf is ignored)."""

    def __init__(self, points, c: float, p: int, leaf: int, domain=None,
                 check_duplicates: bool = False, stream=None, m2l_kernel: str = "auto",
                 algorithm: str = "fmm", levels: int = 0, allocator: str | None = None,
                 translations: str = "fp32", p2p_warps: int = 0, p2p_chunk: int = 0, m2l_stages: int = 0,
                 m2l_split: int = 0):
        self._h = ctypes.c_void_p(0)
        # allocator="torch": the plan's own buffers come from torch's caching allocator
        self._alloc_cbs = _torch_allocator() if allocator == "torch" else None
        pts_ptr, keep = _buf(points, torch.float64)
        n = int(np.shape(points)[0])
        opt = _plan_options(domain, check_duplicates, m2l_kernel, algorithm, levels, self._alloc_cbs,
                            translations, p2p_warps, p2p_chunk, m2l_stages, m2l_split)
        call("imq_plan", pts_ptr, n, float(c), int(p), int(leaf), ctypes.byref(opt), _stream(stream),
             ctypes.byref(self._h))
        del keep
        self.n = n
        self.c = float(c)
        self.p = int(p)
        self.leaf = int(leaf)

    def close(self):
        if self._h and self._h.value:
            _lib.load().imq_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:   # noqa: BLE001 - interpreter shutdown
            pass

    def matvec(self, v, out=None, stream=None):
        """imq_matvec: b = A v (fast method); v is [N] or [nrhs][N], float32 or float64."""
        code = _dtype_code(v)
        tdt = torch.float32 if code == F32 else torch.float64
        nrhs = 1 if len(np.shape(v)) == 1 else int(np.shape(v)[0])
        if out is None:
            out = _like(v, self.n * nrhs, code)
        vp, kv = _buf(v, tdt)
        op, ko = _buf(out, tdt)
        call("imq_matvec", self._h, vp, op, nrhs, code, _stream(stream))
        return out

    def solve(self, f, coef=None, rtol=1e-6, maxit=1000, precond="schwarz", schwarz_nmax=0,
              schwarz_shift=0.0, refine_steps=0, inner_rtol=1e-4, residual="plan", x0=None,
              residual_plan=None, operator="fast_f32", schwarz_fp64=False, coarse_points=0, coarse_gram="auto",
              krylov="cg", gmres_m=0, stream=None, raise_on_failure=False):
        """imq_cg_solve: coef with A coef = f.  Returns (coef, info dict); info["status"] is the
        imq_status name (IMQ_NOT_CONVERGED keeps the best iterate in coef).
        precond: "none", "schwarz" (leaf-neighbourhood patches) or "schwarz2" (the patches plus a
        Galerkin coarse space of tree boxes holding at most coarse_points points).
        krylov: "cg" or "gmres" (restarted GMRES(gmres_m), for numerically indefinite flat shapes)."""
        return self._solve("imq_cg_solve", f, coef, x0, stream, raise_on_failure, None, dict(
            rtol=rtol, maxit=maxit, precond=precond, schwarz_nmax=schwarz_nmax, schwarz_shift=schwarz_shift,
            refine_steps=refine_steps, inner_rtol=inner_rtol, residual=residual, residual_plan=residual_plan,
            operator=operator, schwarz_fp64=schwarz_fp64, coarse_points=coarse_points, coarse_gram=coarse_gram,
            krylov=krylov, gmres_m=gmres_m))

    def _solve(self, entry, f, coef, x0, stream, raise_on_failure, per_problem, kw):
        nrhs = 1 if len(np.shape(f)) == 1 else int(np.shape(f)[0])
        if coef is None:
            coef = _like(f, 0, F64) if x0 is None else (x0.clone() if isinstance(x0, torch.Tensor) else np.array(x0, dtype=np.float64))
        elif x0 is not None:
            raise ValueError("pass either coef or x0")
        o = CgOptions()
        _lib.load().imq_cg_default_options(ctypes.byref(o))
        o.rtol = float(kw["rtol"])
        o.maxit = int(kw["maxit"])
        o.precond = PRECONDS[kw["precond"]]
        o.coarse_points = int(kw.get("coarse_points", 0))
        o.coarse_gram = COARSE_GRAMS[kw.get("coarse_gram", "auto")]
        o.schwarz_nmax = int(kw["schwarz_nmax"])
        o.schwarz_shift = float(kw["schwarz_shift"])
        o.refine_steps = int(kw["refine_steps"])
        o.inner_rtol = float(kw["inner_rtol"])
        o.residual = RESIDUALS[kw["residual"]]
        o.x0_given = 1 if x0 is not None else 0
        rp = kw.get("residual_plan")
        o.residual_plan = rp._h if rp is not None else None
        o.inner_operator = OPERATORS[kw["operator"]]
        o.schwarz_fp64 = 1 if kw["schwarz_fp64"] else 0
        o.krylov = KRYLOVS[kw.get("krylov", "cg")]
        o.gmres_m = int(kw.get("gmres_m", 0))
        info = CgInfo()
        fp, kf = _buf(f, torch.float64)
        cp, kc = _buf(coef, torch.float64)
        lib = _lib.load()
        if per_problem is None:
            st = lib.imq_cg_solve(self._h, fp, cp, nrhs, ctypes.byref(o), ctypes.byref(info), _stream(stream))
        else:
            rel = np.zeros((nrhs, per_problem), dtype=np.float64)
            its = np.zeros((nrhs, per_problem), dtype=np.int32)
            st = lib.imq_cg_solve_batched(self._h, fp, cp, nrhs, ctypes.byref(o), ctypes.byref(info),
                                          ctypes.c_void_p(rel.ctypes.data), ctypes.c_void_p(its.ctypes.data),
                                          _stream(stream))
        msg = lib.imq_last_error().decode()
        out = {"status": _lib.status_name(st), "iterations": info.iterations, "outer_steps": info.outer_steps,
               "max_rel_residual": info.max_rel_residual, "seconds": info.seconds,
               "rel_residual": list(info.rel_residual)[:min(nrhs, 16)], "message": msg}
        if per_problem is not None:
            out["problem_rel_residual"] = rel
            out["problem_iterations"] = its
        # IMQ_NOT_CONVERGED (5) and IMQ_NUMERICAL (6) still return the best iterate and its info
        if st != 0 and (raise_on_failure or st not in (5, 6)):
            raise ImqError(st, entry, msg)
        return coef, out

    def matvec_dc(self, v, out=None, stream=None):
        """imq_matvec_dc: b = (dA/dc) v, dA_ij/dc = -c (r^2 + c^2)^{-3/2}."""
        code = _dtype_code(v)
        tdt = torch.float32 if code == F32 else torch.float64
        nrhs = 1 if len(np.shape(v)) == 1 else int(np.shape(v)[0])
        if out is None:
            out = _like(v, self.n * nrhs, code)
        vp, kv = _buf(v, tdt)
        op, ko = _buf(out, tdt)
        call("imq_matvec_dc", self._h, vp, op, nrhs, code, _stream(stream))
        return out

    PHASES = ("gather", "p2m", "m2m", "m2l", "p2l", "l2l", "l2p_m2p", "p2p", "scatter")

    def matvec_timed(self, v, out=None, stream=None):
        """imq_matvec_timed: (out, {phase: ms}, kernel launches); synchronises the stream."""
        code = _dtype_code(v)
        tdt = torch.float32 if code == F32 else torch.float64
        nrhs = 1 if len(np.shape(v)) == 1 else int(np.shape(v)[0])
        if out is None:
            out = _like(v, self.n * nrhs, code)
        vp, kv = _buf(v, tdt)
        op, ko = _buf(out, tdt)
        ms = (ctypes.c_float * len(self.PHASES))()
        nl = ctypes.c_int32(0)
        call("imq_matvec_timed", self._h, vp, op, nrhs, code, _stream(stream), ms, len(self.PHASES),
             ctypes.byref(nl))
        return out, dict(zip(self.PHASES, list(ms))), int(nl.value)

    def info(self) -> dict:
        inf = PlanInfo()
        call("imq_plan_get_info", self._h, ctypes.byref(inf))
        return {name: getattr(inf, name) for name, _ in PlanInfo._fields_}

    def export_tree(self) -> dict:
        inf = self.info()
        n, nb = inf["n_points"], inf["n_boxes"]
        out = dict(codes=np.empty(n, np.uint32), perm=np.empty(n, np.int64), level=np.empty(nb, np.int32),
                   prefix=np.empty(nb, np.uint32), begin=np.empty(nb, np.int64), end=np.empty(nb, np.int64),
                   parent=np.empty(nb, np.int32), child=np.empty((nb, 4), np.int32))
        ptr = {k: ctypes.c_void_p(v.ctypes.data) for k, v in out.items()}
        call("imq_plan_export_tree", self._h, ptr["codes"], ptr["perm"], ptr["level"], ptr["prefix"],
             ptr["begin"], ptr["end"], ptr["parent"], ptr["child"])
        return out

    def export_list(self, which: str):
        inf = self.info()
        nb = inf["n_boxes"]
        off = np.empty(nb + 1, np.int32)
        call("imq_plan_export_list", self._h, which.encode(), ctypes.c_void_p(off.ctypes.data), None)
        items = np.empty(max(1, int(off[-1])), np.int32)
        call("imq_plan_export_list", self._h, which.encode(), ctypes.c_void_p(off.ctypes.data),
             ctypes.c_void_p(items.ctypes.data))
        return off, items[:int(off[-1])]


class EvalPlan(Plan):
    """imq_plan_eval: one tree over nodes and evaluation targets (interpolant of Eq. (2))."""

    def __init__(self, nodes, targets, c: float, p: int, leaf: int, domain=None, stream=None,
                 m2l_kernel: str = "auto"):
        self._h = ctypes.c_void_p(0)
        np_, kn = _buf(nodes, torch.float64)
        tp_, kt = _buf(targets, torch.float64)
        nn, nt = int(np.shape(nodes)[0]), int(np.shape(targets)[0])
        opt = _plan_options(domain, False, m2l_kernel)
        call("imq_plan_eval", np_, nn, tp_, nt, float(c), int(p), int(leaf), ctypes.byref(opt),
             _stream(stream), ctypes.byref(self._h))
        self.n = nn + nt
        self.n_nodes, self.n_targets = nn, nt
        self.c, self.p, self.leaf = float(c), int(p), int(leaf)

    def _eval(self, name, x, n_in, n_out, out, stream):
        code = _dtype_code(x)
        tdt = torch.float32 if code == F32 else torch.float64
        nrhs = 1 if len(np.shape(x)) == 1 else int(np.shape(x)[0])
        if out is None:
            shape = (n_out,) if nrhs == 1 else (nrhs, n_out)
            out = (torch.empty(shape, dtype=tdt, device=x.device) if isinstance(x, torch.Tensor)
                   else np.empty(shape, dtype=np.float32 if code == F32 else np.float64))
        xp, kx = _buf(x, tdt)
        op, ko = _buf(out, tdt)
        call(name, self._h, xp, op, nrhs, code, _stream(stream))
        return out

    def evaluate(self, coef, out=None, stream=None):
        """P(t_k) = sum_j coef_j phi(|t_k - x_j|)."""
        return self._eval("imq_evaluate", coef, self.n_nodes, self.n_targets, out, stream)

    def evaluate_transpose(self, v, out=None, stream=None):
        """(E^T v)_j = sum_k phi(|t_k - x_j|) v_k."""
        return self._eval("imq_evaluate_transpose", v, self.n_targets, self.n_nodes, out, stream)

    def evaluate_dc(self, coef, out=None, stream=None):
        """sum_j coef_j d phi(|t_k - x_j|)/dc."""
        return self._eval("imq_evaluate_dc", coef, self.n_nodes, self.n_targets, out, stream)


class BatchedPlan(Plan):
    """imq_plan_batched: independent problems (points_b, c_b) in one flattened tree."""

    def __init__(self, points_list, c_list, p: int, leaf: int, domain=None, stream=None,
                 m2l_kernel: str = "auto", translations: str = "fp32", p2p_warps: int = 0, p2p_chunk: int = 0,
                 m2l_stages: int = 0, m2l_split: int = 0):
        self._h = ctypes.c_void_p(0)
        sizes = [int(np.shape(x)[0]) for x in points_list]
        offs = np.zeros(len(sizes) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(sizes)
        if all(isinstance(x, torch.Tensor) and x.is_cuda for x in points_list):
            pts = torch.cat([x.to(torch.float64) for x in points_list]).contiguous()
        else:
            pts = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in points_list]))
        cs = np.ascontiguousarray(np.asarray(c_list, dtype=np.float64))
        pp, kp = _buf(pts, torch.float64)
        opt = _plan_options(domain, False, m2l_kernel, translations=translations, p2p_warps=p2p_warps,
                            p2p_chunk=p2p_chunk, m2l_stages=m2l_stages, m2l_split=m2l_split)
        call("imq_plan_batched", pp, ctypes.c_void_p(offs.ctypes.data), len(sizes),
             ctypes.c_void_p(cs.ctypes.data), int(p), int(leaf), ctypes.byref(opt), _stream(stream),
             ctypes.byref(self._h))
        self.n = int(offs[-1])
        self.offsets = offs
        self.c_list = cs
        self.c = float(cs[0])
        self.p, self.leaf = int(p), int(leaf)

    @property
    def n_problems(self) -> int:
        return len(self.c_list)

    def solve(self, f, coef=None, rtol=1e-6, maxit=1000, precond="schwarz", schwarz_nmax=0,
              schwarz_shift=0.0, refine_steps=0, inner_rtol=1e-4, x0=None, operator="fast_f32",
              schwarz_fp64=False, residual="plan", krylov="cg", gmres_m=0, coarse_points=0, coarse_gram="auto",
              stream=None, raise_on_failure=False):
        """imq_cg_solve_batched: every problem's system at once, per-problem Krylov scalars (CG, or
        GMRES(gmres_m) with a Hessenberg matrix per problem; precond="schwarz2" needs GMRES).
        residual="dense" certifies each problem with its own dense FP64 product.
        info adds "problem_rel_residual" and "problem_iterations" ([nrhs, n_problems])."""
        return self._solve("imq_cg_solve_batched", f, coef, x0, stream, raise_on_failure, self.n_problems, dict(
            rtol=rtol, maxit=maxit, precond=precond, schwarz_nmax=schwarz_nmax, schwarz_shift=schwarz_shift,
            refine_steps=refine_steps, inner_rtol=inner_rtol, residual=residual, residual_plan=None,
            operator=operator, schwarz_fp64=schwarz_fp64, krylov=krylov, gmres_m=gmres_m,
            coarse_points=coarse_points, coarse_gram=coarse_gram))


def dense_matvec(points, c: float, v, out=None, stream=None):
    """imq_dense_matvec: b = A v over all N^2 pairs (the plain product)."""
    code = _dtype_code(v)
    tdt = torch.float32 if code == F32 else torch.float64
    n = int(np.shape(points)[0])
    nrhs = 1 if len(np.shape(v)) == 1 else int(np.shape(v)[0])
    if out is None:
        out = _like(v, n * nrhs, code)
    pp, kp = _buf(points, torch.float64)
    vp, kv = _buf(v, tdt)
    op, ko = _buf(out, tdt)
    call("imq_dense_matvec", pp, n, float(c), vp, op, nrhs, code, _stream(stream))
    return out


def dense_matvec_noalloc(points, c: float, v, out, stream=None):
    """imq_dense_matvec_noalloc: FP32 dense product that allocates no device memory.

    For callers that may not allocate (their memory manager owns the device, or
    the call sits on a path that cannot afford an allocation): points (float64
    [N,2]), v and out (float32 [N]) must be CUDA tensors, N <= 262144.  Calls on
    overlapping streams race on the library's one fixed scratch array.
    """
    n = int(points.shape[0])
    pp, kp = _buf(points, torch.float64)
    vp, kv = _buf(v, torch.float32)
    op, ko = _buf(out, torch.float32)
    call("imq_dense_matvec_noalloc", pp, n, float(c), vp, op, _stream(stream))
    return out


def autotune(points, c, target: float = 1e-6, p_candidates=(8, 10, 12, 14, 16),
             leaf_candidates=(32, 64, 128), nrhs: int = 1, domain=None, m2l_kernel: str = "auto", stream=None,
             v=None):
    """imq_autotune: the measured choice of (p, leaf) for one point set, or for a batch.

    points: [N, 2] float64 (host or CUDA) with a scalar c, or a list of [N_b, 2]
    arrays with a list of c_b (batched plans).  v: optional test vectors
    ([nrhs, N] float32, the caller's point order; imq_autotune_v), else
    SplitMix64 values.  Returns a dict with the choice ("p", "leaf", "rel_err",
    "matvec_ms", "met") and every measured configuration under "tried".
    """
    if isinstance(points, (list, tuple)):
        sizes = [int(np.shape(x)[0]) for x in points]
        if all(isinstance(x, torch.Tensor) and x.is_cuda for x in points):
            pts = torch.cat([x.to(torch.float64) for x in points]).contiguous()
        else:
            pts = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in points]))
        cs = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
    else:
        sizes = [int(np.shape(points)[0])]
        pts = points
        cs = np.array([float(c)], dtype=np.float64)
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    pc = np.ascontiguousarray(np.asarray(p_candidates, dtype=np.int32))
    lc = np.ascontiguousarray(np.asarray(leaf_candidates, dtype=np.int32))
    pp, kp = _buf(pts, torch.float64)
    opt = _plan_options(domain, False, m2l_kernel)
    res = TuneResult()
    args = [pp, ctypes.c_void_p(offs.ctypes.data), len(sizes), ctypes.c_void_p(cs.ctypes.data),
            float(target), ctypes.c_void_p(pc.ctypes.data), len(pc), ctypes.c_void_p(lc.ctypes.data), len(lc),
            int(nrhs)]
    if v is None:
        call("imq_autotune", *args, ctypes.byref(opt), _stream(stream), ctypes.byref(res))
    else:
        if int(np.prod(np.shape(v))) != int(nrhs) * int(offs[-1]):
            raise ValueError("v must hold nrhs x N values")
        vp, kv = _buf(v, torch.float32)
        call("imq_autotune_v", *args, vp, ctypes.byref(opt), _stream(stream), ctypes.byref(res))
    names = {v: k for k, v in TRANSLATIONS.items()}

    def entry(t):
        return {"p": t.p, "leaf": t.leaf, "rel_err": t.rel_err, "matvec_ms": t.matvec_ms,
                "translations": names[t.translations], "p2p_warps": t.p2p_warps, "p2p_chunk": t.p2p_chunk,
                "m2l_stages": t.m2l_stages, "m2l_split": t.m2l_split}

    tried = [entry(res.tried[k]) for k in range(res.n_tried)]
    out = entry(res)
    out.update({"met": bool(res.met), "sampled_rows": res.sampled_rows, "tried": tried})
    return out


def tiles_of(tune: dict) -> dict:
    """Plan keyword arguments (translations and tile shapes) of an autotune result."""
    return {k: tune[k] for k in ("translations", "p2p_warps", "p2p_chunk", "m2l_stages", "m2l_split")}


def sync_check(stream=None) -> None:
    """imq_sync_check: synchronise the stream; raise ImqError(IMQ_TIMEOUT) if a kernel's bounded wait ran out."""
    call("imq_sync_check", _stream(stream))


def version() -> str:
    return _lib.load().imq_version().decode()


__all__ = ["Plan", "EvalPlan", "BatchedPlan", "autotune", "tiles_of", "sync_check", "dense_matvec", "dense_matvec_noalloc", "version", "ImqError", "F32", "F64"]
