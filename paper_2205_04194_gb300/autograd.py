"""Gradient of a held-out validation loss of the IMQ interpolant behind torch.autograd.

The interpolant of Eq. (2) with coefficients from A(c) coef = f (Eq. (4)) is
evaluated at validation points; the loss is the mean squared error there.
The forward pass calls imq_interp_loss_grad, which computes the loss and, by
the adjoint method, its gradient in c and in the data values f entirely in the
library's kernels (two CG solves, evaluation, transpose evaluation and the
two c-derivative products).  This module only marshals arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CgInfo, CgOptions
from .imq import F32, F64, EvalPlan, Plan, _buf, _stream


def cg_options(rtol=1e-10, maxit=2000, precond="schwarz", schwarz_nmax=0, schwarz_fp64=False,
               schwarz_shift=0.0, refine_steps=0, inner_rtol=1e-4, residual="plan",
               operator="fast_f32", coarse_points=0, krylov="cg", gmres_m=0) -> CgOptions:
    o = CgOptions()
    _lib.load().imq_cg_default_options(ctypes.byref(o))
    o.rtol, o.maxit = float(rtol), int(maxit)
    o.precond = {"none": 0, "schwarz": 1, "schwarz2": 2}[precond]
    o.coarse_points = int(coarse_points)
    o.krylov = {"cg": 0, "gmres": 1}[krylov]
    o.gmres_m = int(gmres_m)
    o.schwarz_nmax, o.schwarz_fp64 = int(schwarz_nmax), 1 if schwarz_fp64 else 0
    o.schwarz_shift = float(schwarz_shift)
    o.refine_steps, o.inner_rtol = int(refine_steps), float(inner_rtol)
    o.residual = {"plan": 0, "dense": 1}[residual]
    o.inner_operator = {"fast_f32": 0, "fast_f64": 1, "dense_f64": 2}[operator]
    return o


def interp_loss_grad(train: Plan, evalp: EvalPlan, f, y, dtype=torch.float64, **cg):
    """(loss, dL/dc, dL/df, coef, info) for the interpolant on `train` evaluated by `evalp`."""
    n, nv = train.n, evalp.n_targets
    dev = f.device if isinstance(f, torch.Tensor) else torch.device("cpu")
    df = torch.empty(n, dtype=torch.float64, device=dev)
    coef = torch.empty(n, dtype=torch.float64, device=dev)
    fp, kf = _buf(f, torch.float64)
    yp, ky = _buf(y, torch.float64)
    loss, dc = ctypes.c_double(0.0), ctypes.c_double(0.0)
    info = CgInfo()
    opt = cg_options(**cg)
    code = F64 if dtype == torch.float64 else F32
    lib = _lib.load()
    st = lib.imq_interp_loss_grad(train._h, evalp._h, fp, yp, ctypes.byref(opt), code, ctypes.byref(loss),
                                  ctypes.byref(dc), ctypes.c_void_p(df.data_ptr()), ctypes.c_void_p(coef.data_ptr()),
                                  ctypes.byref(info), _stream(None))
    if st not in (0, 5, 6):   # IMQ_NOT_CONVERGED / IMQ_NUMERICAL keep the best iterates
        raise _lib.ImqError(st, "imq_interp_loss_grad", lib.imq_last_error().decode())
    return loss.value, dc.value, df, coef, {"iterations": info.iterations, "status": _lib.status_name(st),
                                             "max_rel_residual": info.max_rel_residual}


class UnconvergedSolve(RuntimeError):
    """The solves behind a gradient did not reach their tolerance (info attached)."""

    def __init__(self, info):
        self.info = info
        super().__init__(f"interpolation solves did not converge: {info}")


class InterpLoss(torch.autograd.Function):
    """L(c, f) = mean_k (P(t_k) - y_k)^2 with P the IMQ interpolant of (x, f) at shape c.

    apply(c, f, train_points, val_points, y_val, p, leaf, domain, dtype, cg_kwargs, allow_unconverged)
    c: 0-d float64 tensor; f: float64 tensor [N] (CUDA); points float64 [.,2] (CUDA).
    A gradient from solves that stopped short of their tolerance (IMQ_NOT_CONVERGED) or broke
    down (IMQ_NUMERICAL) raises UnconvergedSolve unless allow_unconverged is true; either way the
    solver info of the last forward pass is kept in InterpLoss.last_info.
    """

    last_info = None

    @staticmethod
    def forward(ctx, c, f, train_points, val_points, y_val, p, leaf, domain=None, dtype=torch.float64,
                cg_kwargs=None, allow_unconverged=False):
        cval = float(c.detach().item())
        tp = Plan(train_points, cval, p, leaf, domain=domain)
        ep = EvalPlan(train_points, val_points, cval, p, leaf, domain=domain)
        loss, dc, df, coef, info = interp_loss_grad(tp, ep, f.detach().contiguous(), y_val.contiguous(),
                                                    dtype=dtype, **(cg_kwargs or {}))
        tp.close()
        ep.close()
        InterpLoss.last_info = info
        if info["status"] != "IMQ_OK" and not allow_unconverged:
            raise UnconvergedSolve(info)
        ctx.save_for_backward(torch.tensor(dc, dtype=torch.float64, device=f.device), df)
        return torch.tensor(loss, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, g):
        dc, df = ctx.saved_tensors
        return g * dc, g * df, None, None, None, None, None, None, None, None, None
