"""O3a: Algorithm 1 of the paper, step by step, in FP64 (TEST INFRASTRUCTURE ONLY).

Paper Section 2.2, Algorithm 1 ("given u, computes b = A u"), with the
quantities of the separated form Eq. (13):

    d_{n,m} = eps_m (n-m)!/(n+m)!
    h_{n,m}(X - Z) = P_n^m(cos th_{x-z}) / rho_{x-z}^{n+1}
    j_{n,m}(Y - Z) = P_n^m(cos th_{y-z}) rho_{y-z}^n

under the lift of Eq. (11): X = (x, t/2), Y = (y, -t/2) and the block centre
Z = (z, -t/2) of Eq. (12).  Hence rho_{x-z} = sqrt(|x-z|^2 + t^2),
cos th_{x-z} = t / rho_{x-z}, rho_{y-z} = |y - z|, cos th_{y-z} = 0, and the
azimuths are the planar angles of x - z and y - z (taken as 0 when y = z).

Levels l = 1..L partition the square D into 2^{l+1} x 2^{l+1} blocks.  For a
block p at level l:
  * moments  v_k += j_{n,m}(Y_j - Z) sin(m om_{y_j-z}) u_j,
             w_k += j_{n,m}(Y_j - Z) cos(m om_{y_j-z}) u_j   over y_j in p,
    packed as k = n(n+1)/2 + m (0-based here);
  * far field b_i += d_{n,m} h_{n,m}(X_i - Z) [sin(m om_{x_i-z}) v_k + cos(m om_{x_i-z}) w_k]
    for x_i in the blocks of S_p;
  * S_p at l = 1: the blocks not adjacent to p; at l >= 2: the blocks that are
    children of the neighbours of p's parent (the region not already treated
    at a coarser level) and are not adjacent to p;
  * near field at l = L: b_i += A_ij u_j for x_i in the blocks of NS_p (the
    blocks adjacent to p, p included) and y_j in p.
"""
from __future__ import annotations

import math

import numpy as np

from . import harmonics as H


def _blocks(points, domain, nside):
    x0, y0, s = domain
    bx = np.clip(np.floor((points[:, 0] - x0) / s * nside), 0, nside - 1).astype(np.int64)
    by = np.clip(np.floor((points[:, 1] - y0) / s * nside), 0, nside - 1).astype(np.int64)
    return bx, by


def packed_index(n: int, m: int) -> int:
    """k = n(n+1)/2 + m (the paper's k = n(n+1)/2 + m + 1, 0-based)."""
    return n * (n + 1) // 2 + m


def treecode_matvec(points, t: float, u, M: int, L: int, domain=(0.0, 0.0, 1.0),
                    count_pairs: bool = False):
    pts = np.asarray(points, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    n = pts.shape[0]
    K = (M + 1) * (M + 2) // 2
    b = np.zeros(n)
    d = np.zeros(K)
    for nn in range(M + 1):
        for m in range(nn + 1):
            d[packed_index(nn, m)] = H.neumann(m) * math.factorial(nn - m) / math.factorial(nn + m)
    P0 = H.legendre_table(M, 0.0)              # P_n^m(cos th_{y-z}) with cos th = 0
    x0, y0, s = domain
    far_pairs = 0
    near_pairs = 0
    for lev in range(1, L + 1):
        nside = 2 ** (lev + 1)
        h = s / nside
        bx, by = _blocks(pts, domain, nside)
        key = bx * nside + by
        members = {}
        for i, kk in enumerate(key):
            members.setdefault(int(kk), []).append(i)
        members = {kk: np.array(v) for kk, v in members.items()}
        for kk, src in members.items():
            pbx, pby = divmod(kk, nside)
            z = (x0 + (pbx + 0.5) * h, y0 + (pby + 0.5) * h)
            # moments v, w of block p
            dy = pts[src] - np.array(z)
            rho_y = np.hypot(dy[:, 0], dy[:, 1])
            om_y = np.arctan2(dy[:, 1], dy[:, 0])
            v = np.zeros(K)
            w = np.zeros(K)
            for nn in range(M + 1):
                for m in range(nn + 1):
                    jnm = P0[nn, m] * rho_y ** nn
                    k = packed_index(nn, m)
                    v[k] += np.sum(jnm * np.sin(m * om_y) * u[src])
                    w[k] += np.sum(jnm * np.cos(m * om_y) * u[src])
            # S_p
            sp = []
            if lev == 1:
                for qx in range(nside):
                    for qy in range(nside):
                        if max(abs(qx - pbx), abs(qy - pby)) > 1:
                            sp.append((qx, qy))
            else:
                px, py = pbx // 2, pby // 2
                for ax in range(px - 1, px + 2):
                    for ay in range(py - 1, py + 2):
                        if not (0 <= ax < nside // 2 and 0 <= ay < nside // 2):
                            continue
                        for cx in (2 * ax, 2 * ax + 1):
                            for cy in (2 * ay, 2 * ay + 1):
                                if max(abs(cx - pbx), abs(cy - pby)) > 1:
                                    sp.append((cx, cy))
            tg = [members[q[0] * nside + q[1]] for q in sp if (q[0] * nside + q[1]) in members]
            if not tg:
                continue
            tgt = np.concatenate(tg)
            far_pairs += tgt.size * src.size
            dx = pts[tgt] - np.array(z)
            rho_x = np.sqrt(dx[:, 0] ** 2 + dx[:, 1] ** 2 + t * t)
            om_x = np.arctan2(dx[:, 1], dx[:, 0])
            Px = H.legendre_table(M, t / rho_x)
            acc = np.zeros(tgt.size)
            for nn in range(M + 1):
                for m in range(nn + 1):
                    k = packed_index(nn, m)
                    hnm = Px[:, nn, m] / rho_x ** (nn + 1)
                    acc += d[k] * hnm * (np.sin(m * om_x) * v[k] + np.cos(m * om_x) * w[k])
            b[tgt] += acc
        if lev == L:
            for kk, src in members.items():
                pbx, pby = divmod(kk, nside)
                nb = [members[qx * nside + qy]
                      for qx in range(pbx - 1, pbx + 2) for qy in range(pby - 1, pby + 2)
                      if 0 <= qx < nside and 0 <= qy < nside and (qx * nside + qy) in members]
                tgt = np.concatenate(nb)
                near_pairs += tgt.size * src.size
                ddx = pts[tgt, 0][:, None] - pts[src, 0][None, :]
                ddy = pts[tgt, 1][:, None] - pts[src, 1][None, :]
                b[tgt] += (1.0 / np.sqrt(ddx * ddx + ddy * ddy + t * t)) @ u[src]
    if count_pairs:
        return b, far_pairs, near_pairs
    return b
