"""O3b: FP64 complex fast-multipole reference of the IMQ product.

TEST INFRASTRUCTURE ONLY.

Paper Section 2.2: with X = (x, t/2) and Y = (y, -t/2), phi(|x-y|) =
G(X;Y) = 1/|X-Y| (Eq. (11)), and G is expanded about a centre Z = (z, -t/2)
placed in the sources' plane (Eq. (12)-(13)).  This module keeps that lift
and those centres, and adds the translations of the fast multipole method
(Greengard-Rokhlin, the paper's reference for FMM) so that expansions move
between boxes of the adaptive tree of ``oracle.tree``:

* multipole of box B about Z_B = (centre_B, -c/2): M_n^m = sum_j u_j conj(U_n^m(Y_j - Z_B))
* local of box B about C_B = (centre_B, +c/2):   Phi(X) = sum L_k^l conj(U_k^l(X - C_B))
* M2M  M_n^m(P) = sum_{k,l} M_k^l(Q) conj(U_{n-k}^{m-l}(Z_Q - Z_P))
* M2L  L_k^l(B) = (-1)^k sum_{n,m} M_n^m(S) T_{n+k}^{m+l}(C_B - Z_S)      (V list)
* P2L  L_k^l(B) = sum_j u_j T_k^l(Y_j - C_B)                              (X list)
* L2L  L_j^i(Q) = sum_{k,l} L_k^l(P) conj(U_{k-j}^{l-i}(C_Q - C_P))
* L2P  Phi(X_i) = sum L_k^l conj(U_k^l(X_i - C_B))
* M2P  Phi(X_i) = sum M_n^m(S) T_n^m(X_i - Z_S)                            (W list; the paper's own far-field formula, Eq. (13))
* P2P  b_i += sum_j u_j phi(|x_i - x_j|)                                  (U list; NS_p of Algorithm 1)

U and T are the solid harmonics of ``oracle.harmonics``.  All coefficients are
kept for -n <= m <= n (no symmetry or parity shortcut), so that the vanishing
of the n+m odd multipole terms and of the imaginary part of the result are
checked, not assumed.  Translation matrices are formed per distinct
displacement (one per level and integer offset) and applied with numpy
matrix products.
"""
from __future__ import annotations

import numpy as np

from . import harmonics as H
from .tree import Tree, build_tree


def _flat(p: int, n, m):
    return n * (2 * p + 1) + (m + p)


class _Ops:
    """Translation-matrix factory for truncation order p."""

    def __init__(self, p: int):
        self.p = p
        K = (p + 1) * (2 * p + 1)
        self.K = K
        n_out, m_out, n_in, m_in = [], [], [], []
        for n in range(p + 1):
            for m in range(-n, n + 1):
                for k in range(p + 1):
                    for l in range(-k, k + 1):
                        n_out.append(n); m_out.append(m); n_in.append(k); m_in.append(l)
        self.no = np.array(n_out); self.mo = np.array(m_out)
        self.ni = np.array(n_in); self.mi = np.array(m_in)
        self.fo = _flat(p, self.no, self.mo)
        self.fi = _flat(p, self.ni, self.mi)
        self.cache = {}

    def m2m(self, t):
        """Matrix (out parent (n,m), in child (k,l)) of conj(U_{n-k}^{m-l}(t))."""
        key = ("m2m",) + tuple(t)
        if key in self.cache:
            return self.cache[key]
        p = self.p
        Ut = H.regular(p, np.asarray(t, dtype=np.float64))
        dn = self.no - self.ni
        dm = self.mo - self.mi
        ok = (dn >= 0) & (np.abs(dm) <= dn)
        T = np.zeros((self.K, self.K), dtype=np.complex128)
        T[self.fo[ok], self.fi[ok]] = np.conj(Ut[dn[ok], dm[ok] + p])
        self.cache[key] = T
        return T

    def l2l(self, t):
        """Matrix (out child (j,i), in parent (k,l)) of conj(U_{k-j}^{l-i}(t))."""
        key = ("l2l",) + tuple(t)
        if key in self.cache:
            return self.cache[key]
        p = self.p
        Ut = H.regular(p, np.asarray(t, dtype=np.float64))
        dn = self.ni - self.no
        dm = self.mi - self.mo
        ok = (dn >= 0) & (np.abs(dm) <= dn)
        T = np.zeros((self.K, self.K), dtype=np.complex128)
        T[self.fo[ok], self.fi[ok]] = np.conj(Ut[dn[ok], dm[ok] + p])
        self.cache[key] = T
        return T

    def m2l(self, d):
        """Matrix (out local (k,l), in multipole (n,m)) of (-1)^k T_{n+k}^{m+l}(d)."""
        key = ("m2l",) + tuple(d)
        if key in self.cache:
            return self.cache[key]
        p = self.p
        Td = H.irregular(2 * p, np.asarray(d, dtype=np.float64))
        valid = (np.abs(self.mo) <= self.no) & (np.abs(self.mi) <= self.ni)
        nn = self.no + self.ni
        mm = self.mo + self.mi
        T = np.zeros((self.K, self.K), dtype=np.complex128)
        sign = np.where(self.no % 2 == 0, 1.0, -1.0)
        T[self.fo[valid], self.fi[valid]] = sign[valid] * Td[nn[valid], mm[valid] + 2 * p]
        self.cache[key] = T
        return T


def _mask(p: int) -> np.ndarray:
    m = np.zeros((p + 1, 2 * p + 1), dtype=bool)
    for n in range(p + 1):
        m[n, p - n:p + n + 1] = True
    return m


def fmm_matvec(points, c: float, u, p: int, leaf: int, domain=None, tree: Tree | None = None,
               return_state: bool = False):
    """b ~= A u by the FMM on the adaptive tree; FP64 complex arithmetic."""
    pts = np.asarray(points, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    n = pts.shape[0]
    t = tree if tree is not None else build_tree(pts, leaf, domain)
    ops = _Ops(p)
    K = ops.K
    nb = t.nbox
    cen = t.centres()
    ps = pts[t.perm]
    us = u[t.perm]
    hc = 0.5 * c
    Mp = np.zeros((nb, K), dtype=np.complex128)
    Lc = np.zeros((nb, K), dtype=np.complex128)

    def src3(b, ctr, z):
        sl = slice(int(t.begin[b]), int(t.end[b]))
        v = np.zeros((sl.stop - sl.start, 3))
        v[:, 0] = ps[sl, 0] - ctr[0]
        v[:, 1] = ps[sl, 1] - ctr[1]
        v[:, 2] = z
        return sl, v

    # P2M at leaves (sources and multipole centre both at height -c/2)
    for b in range(nb):
        if t.is_leaf[b] and t.end[b] > t.begin[b]:
            sl, v = src3(b, cen[b], 0.0)
            Ub = H.regular(p, v).reshape(-1, K)
            Mp[b] = us[sl] @ np.conj(Ub)
    # M2M, finest level first
    order = np.argsort(-t.level, kind="stable")
    for b in order:
        if t.is_leaf[b]:
            continue
        for q in t.children(b):
            dz = (cen[q, 0] - cen[b, 0], cen[q, 1] - cen[b, 1], 0.0)
            Mp[b] += ops.m2m(dz) @ Mp[q]
    # M2L over V lists, P2L over X lists
    for b in range(nb):
        for s in t.V[b]:
            d = (cen[b, 0] - cen[s, 0], cen[b, 1] - cen[s, 1], c)
            Lc[b] += ops.m2l(d) @ Mp[s]
        for s in t.X[b]:
            sl, v = src3(s, cen[b], -c)
            Ts = H.irregular(p, v).reshape(-1, K)
            Lc[b] += us[sl] @ Ts
    # L2L, coarsest level first
    for b in np.argsort(t.level, kind="stable"):
        for q in t.children(int(b)):
            dz = (cen[q, 0] - cen[b, 0], cen[q, 1] - cen[b, 1], 0.0)
            Lc[q] += ops.l2l(dz) @ Lc[b]
    # evaluation at leaves
    bs = np.zeros(n, dtype=np.complex128)
    for b in range(nb):
        if not t.is_leaf[b] or t.end[b] == t.begin[b]:
            continue
        sl, v = src3(b, cen[b], 0.0)
        Ub = H.regular(p, v).reshape(-1, K)
        bs[sl] += np.conj(Ub) @ Lc[b]                          # L2P
        for s in t.W[b]:                                       # M2P
            v2 = np.zeros_like(v)
            v2[:, 0] = ps[sl, 0] - cen[s, 0]
            v2[:, 1] = ps[sl, 1] - cen[s, 1]
            v2[:, 2] = c
            bs[sl] += H.irregular(p, v2).reshape(-1, K) @ Mp[s]
        for s in t.U[b]:                                       # P2P
            ss = slice(int(t.begin[s]), int(t.end[s]))
            dx = ps[sl, 0][:, None] - ps[ss, 0][None, :]
            dy = ps[sl, 1][:, None] - ps[ss, 1][None, :]
            bs[sl] += (1.0 / np.sqrt(dx * dx + dy * dy + c * c)) @ us[ss]
    out = np.empty(n, dtype=np.complex128)
    out[t.perm] = bs
    if return_state:
        return out, dict(tree=t, M=Mp.reshape(nb, p + 1, 2 * p + 1),
                         L=Lc.reshape(nb, p + 1, 2 * p + 1), ops=ops)
    return np.real(out)


def multipole_of_points(p: int, centre_xy, src_xy, u) -> np.ndarray:
    """P2M of arbitrary in-plane sources about an in-plane centre (shape (p+1, 2p+1))."""
    src_xy = np.asarray(src_xy, dtype=np.float64)
    v = np.zeros((src_xy.shape[0], 3))
    v[:, 0] = src_xy[:, 0] - centre_xy[0]
    v[:, 1] = src_xy[:, 1] - centre_xy[1]
    return np.tensordot(np.asarray(u, dtype=np.float64), np.conj(H.regular(p, v)), axes=(0, 0))


def evaluate_local(p: int, L, centre_xy, tgt_xy) -> np.ndarray:
    """L2P of a local expansion at in-plane targets (complex result)."""
    tgt_xy = np.asarray(tgt_xy, dtype=np.float64)
    v = np.zeros((tgt_xy.shape[0], 3))
    v[:, 0] = tgt_xy[:, 0] - centre_xy[0]
    v[:, 1] = tgt_xy[:, 1] - centre_xy[1]
    return np.sum(np.conj(H.regular(p, v)) * L[None], axis=(1, 2))


def ops_for(p: int) -> _Ops:
    return _Ops(p)


def odd_mask(p: int) -> np.ndarray:
    """Boolean [n, m+p] mask of the n+|m| odd coefficients inside |m| <= n."""
    m = _mask(p)
    for n in range(p + 1):
        for mm in range(-n, n + 1):
            if (n + abs(mm)) % 2 == 0:
                m[n, mm + p] = False
    return m
