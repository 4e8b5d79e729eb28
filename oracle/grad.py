"""O5: gradient of a held-out validation loss of the IMQ interpolant (TEST INFRASTRUCTURE ONLY).

The interpolant of Eq. (2), P(x) = sum_j coef_j phi_c(|x - x_j|), with coef
solving A(c) coef = f (Eq. (4)), is evaluated at validation points v_k:
P = E(c) coef, E_kj = phi_c(|v_k - x_j|).  The loss is the mean squared error
L = mean_k (P_k - y_k)^2.  With g = (2/N_v)(P - y) and, A being symmetric,
lambda = A^{-1} E^T g:

    dL/df = lambda
    dL/dc = g^T (dE/dc) coef - lambda^T (dA/dc) coef,
    d phi_c / dc = -c / (r^2 + c^2)^{3/2}.

Dense FP64 (Cholesky) for small N; central finite differences check it.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import dense


def loss(train, c: float, f, val, y_val) -> float:
    A = dense.assemble(train, c)
    coef = sla.cho_solve(sla.cho_factor(A, lower=True), np.asarray(f, dtype=np.float64))
    P = dense.evaluate(train, c, coef, val)
    return float(np.mean((P - y_val) ** 2))


def loss_and_grad(train, c: float, f, val, y_val):
    A = dense.assemble(train, c)
    cf = sla.cho_factor(A, lower=True)
    coef = sla.cho_solve(cf, np.asarray(f, dtype=np.float64))
    P = dense.evaluate(train, c, coef, val)
    nv = val.shape[0]
    g = (2.0 / nv) * (P - y_val)
    lam = sla.cho_solve(cf, dense.evaluate_transpose(train, c, g, val))
    dEc = dense.evaluate(train, c, coef, val, deriv=True)
    dAc = dense.matvec_dc(train, c, coef)
    dc = float(g @ dEc - lam @ dAc)
    return float(np.mean((P - y_val) ** 2)), dc, lam
