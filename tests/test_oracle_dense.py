"""Pins for oracle.dense (O1): Eqs. (2), (4), (5) of the paper."""
import math

import numpy as np
import pytest

from oracle import dense, treecode
from paper_2205_04194_gb300 import workloads as W


def test_single_point_and_pair_closed_forms():
    c = 0.37
    assert dense.matvec(np.array([[0.2, 0.9]]), c, np.array([2.5]))[0] == pytest.approx(2.5 / c)
    pts = np.array([[0.0, 0.0], [0.3, 0.4]])       # distance 0.5
    u = np.array([1.0, -2.0])
    b = dense.matvec(pts, c, u)
    a = 1.0 / math.sqrt(0.25 + c * c)
    assert b[0] == pytest.approx(1.0 / c - 2.0 * a, rel=1e-15)
    assert b[1] == pytest.approx(a - 2.0 / c, rel=1e-15)


def test_brute_force_python_loop():
    pts = W.uniform_points(40, 9)
    u = W.random_vector(40, 9)
    c = 0.05
    b = dense.matvec(pts, c, u)
    for i in range(40):
        s = 0.0
        for j in range(40):
            s += u[j] / math.hypot(math.hypot(pts[i, 0] - pts[j, 0], pts[i, 1] - pts[j, 1]), c)
        assert b[i] == pytest.approx(s, rel=1e-13)


def test_symmetry_and_positive_definiteness():
    pts = W.uniform_points(300, 3)
    h = W.mean_nn_spacing(pts)
    A = dense.assemble(pts, 2 * h)
    assert np.array_equal(A, A.T)
    # Micchelli: IMQ matrices of distinct points are positive definite
    assert np.linalg.eigvalsh(A).min() > 0
    np.linalg.cholesky(A)
    g = np.random.default_rng(0)
    u, v = g.standard_normal(300), g.standard_normal(300)
    assert u @ dense.matvec(pts, 2 * h, v) == pytest.approx(v @ dense.matvec(pts, 2 * h, u), rel=1e-12)


def test_large_shape_limit_and_multirhs():
    pts = W.uniform_points(200, 4)
    u = W.random_vector(200, 4, nrhs=3)
    c = 1e7
    b = dense.matvec(pts, c, u)
    assert np.allclose(b, u.sum(axis=1, keepdims=True) / c, rtol=1e-12)
    b1 = dense.matvec(pts, 0.1, u)
    for r in range(3):
        assert np.array_equal(b1[r], dense.matvec(pts, 0.1, u[r]))


def test_rows_evaluate_and_transpose():
    pts = W.uniform_points(500, 5)
    u = W.random_vector(500, 5)
    b = dense.matvec(pts, 0.08, u)
    rows = np.array([0, 17, 499, 250])
    assert np.array_equal(dense.matvec_rows(pts, 0.08, u, rows), b[rows])
    assert np.allclose(dense.evaluate(pts, 0.08, u, pts), b, rtol=1e-14)
    tg = W.uniform_points(70, 6)
    r = W.random_vector(70, 6)
    E = np.array([[1 / math.sqrt((t[0] - s[0]) ** 2 + (t[1] - s[1]) ** 2 + 0.08 ** 2) for s in pts] for t in tg])
    assert np.allclose(dense.evaluate(pts, 0.08, u, tg), E @ u, rtol=1e-13)
    assert np.allclose(dense.evaluate_transpose(pts, 0.08, r, tg), E.T @ r, rtol=1e-13)


def test_dc_kernel_is_derivative_in_c():
    pts = W.uniform_points(300, 7)
    u = W.random_vector(300, 7)
    c, h = 0.1, 1e-5
    fd = (dense.matvec(pts, c + h, u) - dense.matvec(pts, c - h, u)) / (2 * h)
    # central differences: O(h^2) truncation, O(eps/h) rounding
    assert np.max(np.abs(dense.matvec_dc(pts, c, u) - fd)) < 1e-6 * np.max(np.abs(fd))


def test_dense_agrees_with_independent_treecode():
    # Algorithm 1 is a different computation of the same product
    pts = W.halton_points(3000)
    u = W.random_vector(3000, 6)
    b = dense.matvec(pts, 1.0, u)
    bt = treecode.treecode_matvec(pts, 1.0, u, 20, 2)
    assert np.max(np.abs(b - bt)) / np.max(np.abs(b)) < 1e-13
