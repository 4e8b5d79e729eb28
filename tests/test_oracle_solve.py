"""Pins for oracle.solve (O2) and oracle.grad (O5)."""
import numpy as np
import pytest

from oracle import dense, grad, solve
from paper_2205_04194_gb300 import workloads as W


def test_cholesky_interpolant_reproduces_data():
    # Eq. (3): P_f(x_i) = f_i at the nodes
    pts = W.uniform_points(800, 1)
    c = 2 * W.mean_nn_spacing(pts)
    f = W.franke(pts)
    coef = solve.cholesky(pts, c, f)
    assert solve.true_relres(pts, c, coef, f) < 1e-12
    assert np.allclose(dense.evaluate(pts, c, coef, pts), f, atol=1e-11)


def test_cg_reaches_cholesky_solution_well_conditioned():
    pts = W.uniform_points(600, 2)
    c = 2 * W.mean_nn_spacing(pts)
    f = W.sincos_noisy(pts, 2)
    mv = lambda x: dense.matvec(pts, c, x)
    x, it, hist, ok = solve.cg(mv, f, 1e-10, 5000)
    assert ok and hist[-1] <= 1e-10
    assert solve.true_relres(pts, c, x, f) < 1e-9
    # the recursive residual history is non-increasing in the A-norm sense; check the end points
    assert hist[0] == pytest.approx(1.0)


def test_schwarz_pcg_beats_cg():
    pts = W.uniform_points(2000, 1)
    c = 0.1
    f = W.franke(pts)
    mv = lambda x: dense.matvec(pts, c, x)
    M = solve.schwarz(pts, c, 32)
    x, it, hist, ok = solve.cg(mv, f, 1e-10, 300, precond=M)
    assert ok and it < 100
    assert solve.true_relres(pts, c, x, f) < 1e-9
    _, it_cg, hist_cg, ok_cg = solve.cg(mv, f, 1e-10, 300)
    assert (not ok_cg) or it_cg > 3 * it


def test_gradient_matches_central_differences():
    tr = W.uniform_points(250, 5, stream=0)
    va = W.uniform_points(60, 5, stream=1)
    f = W.gaussian_bump(tr)
    y = W.gaussian_bump(va)
    c = 0.3
    L, dc, lam = grad.loss_and_grad(tr, c, f, va, y)
    h = 1e-5
    fd = (grad.loss(tr, c + h, f, va, y) - grad.loss(tr, c - h, f, va, y)) / (2 * h)
    assert dc == pytest.approx(fd, rel=1e-4, abs=1e-10)
    for j in (0, 17, 111, 249):
        fp, fm = f.copy(), f.copy()
        fp[j] += h
        fm[j] -= h
        fdj = (grad.loss(tr, c, fp, va, y) - grad.loss(tr, c, fm, va, y)) / (2 * h)
        assert lam[j] == pytest.approx(fdj, rel=1e-4, abs=1e-9)
