"""GPU conjugate-gradient solve vs the FP64 oracle.

Parity on the solve is defined on residuals (the interpolant reproduces the
data at the nodes, Eq. (3)): the true relative residual ||f - A coef|| / ||f||
of the GPU coefficients, measured with the oracle's dense FP64 product, must
meet the requested tolerance.  Coefficients themselves are compared with the
oracle's Cholesky solution only for information (they can differ by ~kappa*tol).
"""
import numpy as np
import pytest

from gpu_util import cuda, host, need_gpu
from oracle import solve as OS
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _imq():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    return imq


def _well_conditioned(n=2000, seed=1):
    pts = W.uniform_points(n, seed)
    c = 2.0 * W.mean_nn_spacing(pts)
    return pts, c, W.franke(pts)


def test_cg_unpreconditioned_fp32_operator():
    imq = _imq()
    pts, c, f = _well_conditioned()
    plan = imq.Plan(cuda(pts), c, 12, 32)
    coef, info = plan.solve(cuda(f), rtol=1e-6, maxit=20000, precond="none", residual="dense")
    assert info["status"] == "IMQ_OK", info
    x = host(coef)
    assert OS.true_relres(pts, c, x, f) <= 1e-6
    assert info["max_rel_residual"] <= 1e-6


def test_schwarz_pcg_needs_far_fewer_iterations():
    imq = _imq()
    pts, c, f = _well_conditioned()
    plan = imq.Plan(cuda(pts), c, 12, 32)
    _, i0 = plan.solve(cuda(f), rtol=1e-6, maxit=20000, precond="none")
    coef, i1 = plan.solve(cuda(f), rtol=1e-6, maxit=20000, precond="schwarz", schwarz_nmax=128,
                          residual="dense")
    assert i1["status"] == "IMQ_OK", i1
    assert i1["iterations"] * 5 < i0["iterations"]
    assert OS.true_relres(pts, c, host(coef), f) <= 1e-6


def test_plain_2k_fp64_to_1e10():
    imq = _imq()
    wl = W.plain_2k()
    plan = imq.Plan(cuda(wl.points), wl.c, wl.p, wl.leaf, domain=wl.domain)
    coef, info = plan.solve(cuda(wl.f), rtol=1e-10, maxit=3000, precond="schwarz", schwarz_nmax=160,
                            schwarz_fp64=True, operator="dense_f64", residual="dense")
    assert info["status"] == "IMQ_OK", info
    assert OS.true_relres(wl.points, wl.c, host(coef), wl.f) <= 1e-10


def test_refinement_fp32_inner_fp64_residual():
    imq = _imq()
    pts, c, f = _well_conditioned(4000, 3)
    f = W.sincos_noisy(pts, 3)
    plan = imq.Plan(cuda(pts), c, 12, 32)
    coef, info = plan.solve(cuda(f), rtol=1e-8, maxit=5000, precond="schwarz", refine_steps=8,
                            inner_rtol=1e-5, residual="dense")
    assert info["status"] == "IMQ_OK", info
    assert info["outer_steps"] >= 2
    assert OS.true_relres(pts, c, host(coef), f) <= 1e-8


def test_not_converged_returns_best_iterate_and_info():
    imq = _imq()
    pts, c, f = _well_conditioned(1500, 4)
    plan = imq.Plan(cuda(pts), c, 10, 32)
    coef, info = plan.solve(cuda(f), rtol=1e-12, maxit=3, precond="none")
    assert info["status"] == "IMQ_NOT_CONVERGED"
    assert info["iterations"] == 3
    r = OS.true_relres(pts, c, host(coef), f)
    assert 0 < r < 1.0 and info["max_rel_residual"] == pytest.approx(r, rel=1e-3)


def test_multiple_rhs_host_buffers_and_determinism():
    imq = _imq()
    pts, c, f0 = _well_conditioned(2500, 5)
    F = np.stack([f0, W.trig_sum(pts, 5, 1)])
    plan = imq.Plan(cuda(pts), c, 12, 32)
    # 1e-7 is below what one pass on the FP32 operator certifies: refine with the dense FP64 residual
    kw = dict(rtol=1e-7, maxit=5000, refine_steps=4, residual="dense")
    a, ia = plan.solve(F, **kw)                              # numpy in, numpy out
    b, ib = plan.solve(cuda(F), **kw)
    assert ia["status"] == "IMQ_OK" and isinstance(a, np.ndarray), ia
    assert np.array_equal(a, host(b))                        # bit-reproducible
    for r in range(2):
        assert OS.true_relres(pts, c, a[r], F[r]) <= 1e-7


def test_flat_shape_breakdown_returns_best_iterate():
    """c = 30 x the mean nearest-neighbour spacing: A is SPD but numerically
    singular, the FP32 product is not positive on every direction, and CG can
    break down.  The solve must then restart from its best iterate, never report
    a breakdown as a NaN, and report the true residual of the iterate it returns."""
    imq = _imq()
    pts = W.uniform_points(4000, 6)
    c = 30.0 * W.mean_nn_spacing(pts)
    f = W.franke(pts)
    plan = imq.Plan(cuda(pts), c, 12, 64)
    coef, info = plan.solve(cuda(f), rtol=1e-6, maxit=400, precond="schwarz", schwarz_nmax=128,
                            schwarz_shift=1e-5, residual="dense")
    assert info["status"] in ("IMQ_OK", "IMQ_NOT_CONVERGED"), info
    r = OS.true_relres(pts, c, host(coef), f)
    assert np.isfinite(r) and r < 0.1, (r, info)
    assert info["max_rel_residual"] == pytest.approx(r, rel=1e-2, abs=1e-12)
