"""Restarted GMRES as the inner Krylov method of imq_cg_solve, against the FP64 oracle.

Parity of a solve is defined on residuals (the interpolant reproduces the data
at the nodes, Section 2, Eq. (3)): the returned coefficients must give a true
relative residual ||f - A coef|| / ||f|| at or below the requested tolerance,
measured with the oracle's dense product O1.  At the full 1M clustered size the
oracle computes sampled rows of the residual, which must match the GPU's FP64
residual rows and estimate the same norm.
"""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu
from oracle import dense as OD
from oracle import solve as OS
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", ["schwarz", "schwarz2"])
def test_gmres_uniform_meets_1e10_against_the_oracle(precond):
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts = W.uniform_points(3000, 11)
    c = 2.0 * W.mean_nn_spacing(pts)
    f = np.sin(6 * pts[:, 0]) * np.cos(4 * pts[:, 1])
    plan = imq.Plan(cuda(pts), c, 12, 32, domain=(0.0, 0.0, 1.0))
    coef, info = plan.solve(cuda(f), rtol=1e-10, maxit=2000, precond=precond, coarse_points=128,
                            residual="dense", krylov="gmres", gmres_m=30)
    assert info["status"] == "IMQ_OK", info
    r = OS.true_relres(pts, c, host(coef), f)
    assert r <= 1e-10, r
    assert info["max_rel_residual"] == pytest.approx(r, rel=1e-3, abs=1e-13)


def test_gmres_reaches_1e6_on_the_flat_clustered_analogue():
    """The 1M clustered configuration scaled to 5,004 points (c scaled with the spacing, c/h ~ 40
    in the clusters): the FP32 fast operator with the two-level preconditioner; GMRES meets 1e-6
    on the oracle's residual."""
    need_gpu()
    from paper_2205_04194_gb300 import imq
    scale = 0.005
    pts = W.clustered_points(int(round(87_500 * scale)), 8, int(round(300_000 * scale)), 0.03, 3)
    c = 0.01 / np.sqrt(scale)
    f = W.franke(pts)
    plan = imq.Plan(cuda(pts), c, 12, 64, domain=(0.0, 0.0, 1.0))
    coef, info = plan.solve(cuda(f), rtol=1e-6, maxit=1000, precond="schwarz2", coarse_points=256,
                            schwarz_shift=1e-4, residual="dense", krylov="gmres", gmres_m=40)
    assert info["status"] == "IMQ_OK", info
    assert OS.true_relres(pts, c, host(coef), f) <= 1e-6


def test_gmres_full_size_clustered_1m_metric_solve():
    """The metric solve as the benchmark runs it (1M clustered points, c = 0.01, p = 12, leaf 64,
    two-level Schwarz, shift 1e-4 / c, GMRES(40)): IMQ_OK at 1e-6, certified by the FP64 fast
    product at p = 16 and, on 1024 sampled rows, by the oracle."""
    need_gpu()
    import torch
    from paper_2205_04194_gb300 import imq
    wl = W.clustered_1m(p=12)
    d_pts = cuda(wl.points)
    f = cuda(wl.f)
    plan = imq.Plan(d_pts, wl.c, 12, wl.leaf, domain=wl.domain)
    coef, info = plan.solve(f, rtol=1e-6, maxit=200, precond="schwarz2", coarse_points=1024,
                            schwarz_shift=1e-4, krylov="gmres", gmres_m=40)
    assert info["status"] == "IMQ_OK", info
    p16 = imq.Plan(d_pts, wl.c, 16, wl.leaf, domain=wl.domain)
    r16 = host(f - p16.matvec(coef))
    fn = float(np.linalg.norm(wl.f))
    assert np.linalg.norm(r16) / fn <= 1e-6
    rows = np.random.default_rng(5).choice(wl.n, 1024, replace=False)
    r_or = wl.f[rows] - OD.matvec_rows(wl.points, wl.c, host(coef), rows)
    # the oracle's residual rows and the GPU's agree to a few per cent of the residual itself ...
    assert np.linalg.norm(r_or - r16[rows]) <= 0.05 * np.linalg.norm(r_or)
    # ... and the sampled estimate of ||f - A coef|| / ||f|| meets the tolerance
    est = np.sqrt(wl.n / rows.size) * np.linalg.norm(r_or) / fn
    assert est <= 1e-6, est
    torch.cuda.synchronize()


def test_gmres_batched_meets_1e9_on_every_problem_against_the_oracle():
    """Per-problem GMRES on a batched plan (three problems of different size, c = 2h each, as in the
    batched CG tests), dense FP64 residuals and FP64 refinement: each problem's coefficients are
    certified by the oracle, and each problem needs about as many iterations as the same solve on
    its own single plan (the batched product equals the per-problem products)."""
    need_gpu()
    from paper_2205_04194_gb300 import imq
    sizes = [900, 2000, 3100]
    pts = [W.uniform_points(n, 31, stream=k) for k, n in enumerate(sizes)]
    cs = [2.0 * W.mean_nn_spacing(x) for x in pts]
    fs = [np.sin(6 * x[:, 0]) * np.cos(4 * x[:, 1]) for x in pts]
    kw = dict(rtol=1e-9, maxit=4000, precond="schwarz", residual="dense", refine_steps=10, inner_rtol=1e-5,
              krylov="gmres", gmres_m=40)
    bp = imq.BatchedPlan([cuda(x) for x in pts], cs, 12, 32, domain=(0.0, 0.0, 1.0))
    coef, info = bp.solve(cuda(np.concatenate(fs)), **kw)
    assert info["status"] == "IMQ_OK", info
    coef = host(coef)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for k in range(len(sizes)):
        r = OS.true_relres(pts[k], cs[k], coef[offs[k]:offs[k + 1]], fs[k])
        assert r <= 1e-9, (k, r)
        assert info["problem_rel_residual"][0, k] == pytest.approx(r, rel=1e-2, abs=1e-12)
        sp = imq.Plan(cuda(pts[k]), cs[k], 12, 32, domain=(0.0, 0.0, 1.0))
        _, i1 = sp.solve(cuda(fs[k]), **kw)
        assert i1["status"] == "IMQ_OK", i1
        its = int(info["problem_iterations"][0, k])
        assert 0.5 * i1["iterations"] <= its <= 1.5 * i1["iterations"] + 5, (k, its, i1["iterations"])
        sp.close()
    bp.close()


def test_gmres_rejects_bad_options():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts = W.uniform_points(500, 1)
    plan = imq.Plan(cuda(pts), 0.05, 8, 32, domain=(0.0, 0.0, 1.0))
    with pytest.raises(imq.ImqError) as e:
        plan.solve(cuda(np.ones(500)), krylov="gmres", gmres_m=201, raise_on_failure=True)
    assert e.value.status == 1
