"""Conditioning of the clustered metric configuration, reproduced in FP64 on a small analogue.

The 1M clustered workload (c = 0.01, eight sigma = 0.03 clusters) is scaled by
0.005 in every count (5,004 points, same generator and seed) and c by
1/sqrt(0.005), so the shape-to-spacing ratio inside the clusters is the same.
Everything here is the FP64 oracle (dense assembly, eigendecomposition, CG):

* the FP64-assembled A is numerically indefinite (its rounding errors exceed
  its smallest eigenvalues), yet a residual below 1e-6 is reachable in FP64
  with a coefficient vector of modest norm (a spectrally regularised solve);
* CG with the one-level Schwarz preconditioner stalls near 1e-5;
* the two-level (balancing) Schwarz preconditioner with a Galerkin coarse space
  of leaf indicators reaches 1e-6 (the paper: Section 4, a preconditioner as
  future work; Section 1, preconditioned iterations after Beatson et al.).
"""
import numpy as np
import pytest

from oracle import dense, solve
from paper_2205_04194_gb300 import workloads as W

SCALE = 0.005


@pytest.fixture(scope="module")
def analogue():
    pts = W.clustered_points(int(round(87_500 * SCALE)), 8, int(round(300_000 * SCALE)), 0.03, 3)
    c = 0.01 / np.sqrt(SCALE)
    return pts, c, W.franke(pts)


def test_fp64_matrix_is_indefinite_yet_1e6_is_reachable(analogue):
    pts, c, f = analogue
    assert pts.shape[0] == 5004
    A = dense.assemble(pts, c)
    lam, Q = np.linalg.eigh(A)
    # positive definite in exact arithmetic (distinct points), indefinite after FP64 rounding
    assert (lam < 0).sum() > 1000 and lam.min() < 0 and lam.max() > 1e4
    # x = sum_k lam_k / (lam_k^2 + mu) (q_k . f) q_k: residual below 1e-6 with |x| < |f|
    fh = Q.T @ f
    x = Q @ (lam / (lam ** 2 + 1e-10) * fh)
    assert solve.true_relres(pts, c, x, f) < 1e-6
    assert np.linalg.norm(x) < np.linalg.norm(f)


def test_one_level_schwarz_stalls_two_level_reaches_1e6(analogue):
    pts, c, f = analogue
    mv = lambda v: dense.matvec(pts, c, v)
    M1 = solve.schwarz(pts, c, 64, delta=1e-9 / c, domain=(0.0, 0.0, 1.0))
    _, it1, h1, ok1 = solve.cg(mv, f, 1e-6, 300, precond=M1)
    assert not ok1 and min(h1) > 5e-6
    M2, Z, _ = solve.two_level(pts, c, 64, domain=(0.0, 0.0, 1.0))
    x, it2, h2, ok2 = solve.cg(mv, f, 1e-6, 300, precond=M2)
    assert ok2 and it2 < 150
    assert solve.true_relres(pts, c, x, f) <= 1e-6
    assert Z.shape[1] > 150   # one coarse vector per leaf


def test_two_level_is_symmetric_and_exact_on_the_coarse_space():
    # c small enough that the patch solves (which amplify rounding by up to 1/(delta c)) stay tame
    pts = W.clustered_points(150, 4, 300, 0.05, 9)
    c = 0.01
    A = dense.assemble(pts, c)
    P, Z, E = solve.two_level(pts, c, 32, coarse_leaf=64, domain=(0.0, 0.0, 1.0))
    n = pts.shape[0]
    Pm = np.stack([P(e) for e in np.eye(n)], axis=1)
    assert np.linalg.norm(Pm - Pm.T) <= 1e-10 * np.linalg.norm(Pm)
    # Galerkin: E = Z^T A Z; z = Z y whenever r = A Z y
    np.testing.assert_allclose(E, Z.T @ A @ Z, rtol=1e-12)
    y = np.random.default_rng(1).standard_normal(Z.shape[1])
    np.testing.assert_allclose(P(A @ (Z @ y)), Z @ y, rtol=0, atol=1e-8 * np.abs(Z @ y).max())
