"""GPU c-derivative products, off-node evaluation and the validation-loss gradient vs the FP64 oracle."""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu, rel2
from oracle import dense, grad
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _imq():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    return imq


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_matvec_dc_vs_oracle(kind):
    import torch
    imq = _imq()
    pts = W.uniform_points(3000, 2) if kind == "uniform" else W.clustered_points(600, 8, 2500, 0.03, 3)
    c = 0.03 if kind == "uniform" else 0.01
    v = W.random_vector(pts.shape[0], 2)
    ref = dense.matvec_dc(pts, c, v)
    plan = imq.Plan(cuda(pts), c, 14, 32)
    b64 = host(plan.matvec_dc(cuda(v)))
    b32 = host(plan.matvec_dc(cuda(v, torch.float32)))
    assert rel2(b64, ref) < 1e-7
    assert rel2(b32, ref) < 2e-6


def test_evaluate_transpose_and_dc_vs_oracle():
    import torch
    imq = _imq()
    nodes = W.uniform_points(2500, 3)
    tg = W.uniform_points(700, 4)
    c = 0.05
    coef = W.random_vector(2500, 5)
    r = W.random_vector(700, 6)
    ep = imq.EvalPlan(cuda(nodes), cuda(tg), c, 14, 32, domain=(0.0, 0.0, 1.0))
    assert rel2(host(ep.evaluate(cuda(coef))), dense.evaluate(nodes, c, coef, tg)) < 1e-7
    assert rel2(host(ep.evaluate(cuda(coef, torch.float32))), dense.evaluate(nodes, c, coef, tg)) < 2e-6
    assert rel2(host(ep.evaluate_transpose(cuda(r))), dense.evaluate_transpose(nodes, c, r, tg)) < 1e-7
    assert rel2(host(ep.evaluate_dc(cuda(coef))), dense.evaluate(nodes, c, coef, tg, deriv=True)) < 1e-7
    # evaluating at the nodes themselves reproduces the product
    ep2 = imq.EvalPlan(cuda(nodes), cuda(nodes[:100]), c, 14, 32)
    assert rel2(host(ep2.evaluate(cuda(coef))), dense.matvec(nodes, c, coef)[:100]) < 1e-7


def _grad_case():
    tr = W.uniform_points(500, 5, stream=0)
    va = W.uniform_points(120, 5, stream=1)
    return tr, va, W.gaussian_bump(tr), W.gaussian_bump(va), 0.15


def test_gradient_matches_dense_fp64_oracle():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import autograd as AG, imq
    tr, va, f, y, c = _grad_case()
    L0, dc0, lam0 = grad.loss_and_grad(tr, c, f, va, y)
    tp = imq.Plan(cuda(tr), c, 16, 16)
    ep = imq.EvalPlan(cuda(tr), cuda(va), c, 16, 16)
    cg = dict(rtol=1e-13, maxit=4000, operator="dense_f64", residual="dense", schwarz_fp64=True,
              schwarz_nmax=160)
    loss, dc, df, coef, info = AG.interp_loss_grad(tp, ep, cuda(f), cuda(y), dtype=torch.float64, **cg)
    assert loss == pytest.approx(L0, rel=1e-6)
    assert dc == pytest.approx(dc0, rel=1e-4)
    assert rel2(host(df), lam0) < 1e-4


def test_autograd_function_and_central_differences():
    import torch
    need_gpu()
    from paper_2205_04194_gb300 import autograd as AG
    tr, va, f, y, c = _grad_case()
    cg = dict(rtol=1e-13, maxit=4000, operator="dense_f64", residual="dense", schwarz_fp64=True,
              schwarz_nmax=160)
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    ft = cuda(f).requires_grad_(True)
    L = AG.InterpLoss.apply(ct, ft, cuda(tr), cuda(va), cuda(y), 16, 16, None, torch.float64, cg)
    L.backward()
    h = 1e-5

    def loss_at(cv, fv):
        return AG.InterpLoss.apply(torch.tensor(cv, dtype=torch.float64), fv, cuda(tr), cuda(va), cuda(y),
                                   16, 16, None, torch.float64, cg).item()
    fd = (loss_at(c + h, cuda(f)) - loss_at(c - h, cuda(f))) / (2 * h)
    assert ct.grad.item() == pytest.approx(fd, rel=1e-3)
    for j in (3, 250):
        fp, fm = f.copy(), f.copy()
        fp[j] += h
        fm[j] -= h
        fdj = (loss_at(c, cuda(fp)) - loss_at(c, cuda(fm))) / (2 * h)
        assert ft.grad[j].item() == pytest.approx(fdj, rel=1e-3, abs=1e-9)
