"""O2: FP64 solves of the interpolation system A coef = f (TEST INFRASTRUCTURE ONLY).

Paper Section 2, Eq. (3)-(4): the interpolant reproduces the data at the
nodes, i.e. A coef = f with the dense symmetric IMQ matrix A.  The paper
states (Section 1, Section 2) that iterative methods are the practical solver
and that a preconditioner is one way to make them efficient, and leaves the
solver to future work (Section 4).  The oracle therefore offers:

* ``cholesky``: the exact solution of small systems by dense Cholesky
  (scipy ``cho_factor``; succeeds only when A is numerically positive definite);
* ``cg``: conjugate gradients from x0 = 0 (or a given x0) with the rule
  ||r_k||_2 <= rtol ||f||_2 on the recursive residual;
* ``schwarz``: the symmetric additive Schwarz preconditioner
  z = sum_b R_b^T (A_{N(b)} + delta I)^{-1} R_b r, where N(b) is the set of
  points of leaf b and of the leaves adjacent to it (its U list);
* ``two_level``: ``schwarz`` plus a Galerkin coarse space of leaf indicators,
  in the balancing form z = (I - QA) M1 (I - AQ) r + Q r, Q = Z (Z^T A Z)^{-1} Z^T;
* ``true_relres``: ||f - A coef||_2 / ||f||_2 with the dense FP64 product.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import dense
from .tree import build_tree


def cholesky(points, c: float, f):
    A = dense.assemble(points, c)
    cf = sla.cho_factor(A, lower=True)
    return sla.cho_solve(cf, np.asarray(f, dtype=np.float64))


def true_relres(points, c: float, coef, f) -> float:
    r = np.asarray(f, dtype=np.float64) - dense.matvec(points, c, coef)
    return float(np.linalg.norm(r) / np.linalg.norm(f))


def cg(matvec, f, rtol: float, maxit: int, x0=None, precond=None):
    """(P)CG; returns (x, iterations, history of ||r||/||f||, converged)."""
    f = np.asarray(f, dtype=np.float64)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    r = f - matvec(x) if x0 is not None else f.copy()
    nf = np.linalg.norm(f)
    z = precond(r) if precond is not None else r
    p = z.copy()
    rz = float(r @ z)
    hist = [np.linalg.norm(r) / nf]
    if hist[-1] <= rtol:
        return x, 0, hist, True
    for it in range(1, maxit + 1):
        q = matvec(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        hist.append(np.linalg.norm(r) / nf)
        if hist[-1] <= rtol:
            return x, it, hist, True
        z = precond(r) if precond is not None else r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist, False


def schwarz(points, c: float, leaf: int, delta: float = 0.0, domain=None, tree=None):
    """Additive Schwarz over leaf neighbourhood patches; returns r -> z."""
    pts = np.asarray(points, dtype=np.float64)
    t = tree if tree is not None else build_tree(pts, leaf, domain)
    patches = []
    for b in range(t.nbox):
        if not t.is_leaf[b] or t.end[b] == t.begin[b]:
            continue
        idx = np.concatenate([t.perm[int(t.begin[s]):int(t.end[s])] for s in t.U[b]])
        Ab = dense.assemble(pts[idx], c)
        if delta:
            Ab[np.diag_indices_from(Ab)] += delta
        patches.append((idx, sla.cho_factor(Ab, lower=True)))

    def apply(r):
        z = np.zeros_like(r)
        for idx, cf in patches:
            z[idx] += sla.cho_solve(cf, r[idx])
        return z

    return apply


def two_level(points, c: float, leaf: int, coarse_leaf: int | None = None, delta: float = 1e-9, domain=None):
    """Two-level additive Schwarz in its balancing (deflated) form; returns (r -> z, Z, E).

    The paper leaves the preconditioner to future work (Section 4) and names
    preconditioned iterative solvers (Section 1, Beatson et al.).  The one-level
    method is ``schwarz``: local solves on leaf neighbourhood patches.  The
    second level adds a Galerkin coarse space: Z holds the indicator vector of
    every leaf of the tree with ``coarse_leaf`` points per leaf (default: the
    fine leaves), E = Z^T A Z, Q = Z E^{-1} Z^T, and

        z = (I - Q A) M1 (I - A Q) r + Q r

    with M1 the one-level operator.  This is symmetric, and exact on the
    coarse space (z = Z y whenever r = A Z y).  Patch and coarse matrices are
    inverted through their eigendecomposition with eigenvalues clamped below
    at ``delta`` (relative to 1/c for the patches, to the largest eigenvalue for
    E), because both are numerically singular for flat shapes.
    """
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    t = build_tree(pts, leaf, domain)
    A = dense.assemble(pts, c)
    patches = []
    for b in range(t.nbox):
        if not t.is_leaf[b] or t.end[b] == t.begin[b]:
            continue
        idx = np.concatenate([t.perm[int(t.begin[s]):int(t.end[s])] for s in t.U[b]])
        w, V = np.linalg.eigh(A[np.ix_(idx, idx)])
        patches.append((idx, np.maximum(w, delta / c), V))
    tc = t if coarse_leaf is None else build_tree(pts, coarse_leaf, domain)
    cols = []
    for b in range(tc.nbox):
        if tc.is_leaf[b] and tc.end[b] > tc.begin[b]:
            v = np.zeros(n)
            v[tc.perm[int(tc.begin[b]):int(tc.end[b])]] = 1.0
            cols.append(v)
    Z = np.stack(cols, axis=1)
    E = Z.T @ (A @ Z)
    we, Ve = np.linalg.eigh(E)
    we = np.maximum(we, delta * we.max())

    def M1(r):
        z = np.zeros_like(r)
        for idx, w, V in patches:
            z[idx] += V @ ((V.T @ r[idx]) / w)
        return z

    def Q(r):
        return Z @ (Ve @ ((Ve.T @ (Z.T @ r)) / we))

    def apply(r):
        y = Q(r)
        z = M1(r - A @ y)
        return z - Q(A @ z) + y

    return apply, Z, E
