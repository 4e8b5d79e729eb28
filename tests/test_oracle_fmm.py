"""Pins for oracle.fmm (O3b) and oracle.treecode (O3a): Section 2.2 of the paper."""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import dense, fmm, treecode
from oracle import harmonics as H
from oracle import tree as T
from paper_2205_04194_gb300 import workloads as W


def test_single_leaf_is_the_dense_product():
    pts = W.uniform_points(150, 1)
    u = W.random_vector(150, 1)
    b = fmm.fmm_matvec(pts, 0.05, u, 6, leaf=1000)
    assert np.allclose(b, dense.matvec(pts, 0.05, u), rtol=1e-13, atol=1e-12)


def test_m2m_is_exact():
    # P2M at the children, then M2M, equals P2M at the parent (the translation is exact)
    g = np.random.default_rng(0)
    p = 10
    ops = fmm.ops_for(p)
    h = 0.2
    parent = np.array([0.3, 0.6])
    Mp = np.zeros((p + 1, 2 * p + 1), dtype=complex)
    allpts, allu = [], []
    for qx in (-1, 1):
        for qy in (-1, 1):
            cc = parent + np.array([qx, qy]) * h / 4
            pts = cc + g.uniform(-h / 4, h / 4, size=(25, 2))
            u = g.standard_normal(25)
            Mc = fmm.multipole_of_points(p, cc, pts, u)
            Mp += (ops.m2m((cc[0] - parent[0], cc[1] - parent[1], 0.0)) @ Mc.ravel()).reshape(Mp.shape)
            allpts.append(pts)
            allu.append(u)
    direct = fmm.multipole_of_points(p, parent, np.concatenate(allpts), np.concatenate(allu))
    assert np.max(np.abs(Mp - direct)) < 1e-13 * np.max(np.abs(direct))


def test_l2l_is_exact():
    g = np.random.default_rng(1)
    p = 9
    ops = fmm.ops_for(p)
    L = g.standard_normal((p + 1, 2 * p + 1)) + 1j * g.standard_normal((p + 1, 2 * p + 1))
    for n in range(p + 1):                   # make it a real-valued field: L_n^{-m} = (-1)^m conj(L_n^m)
        L[n, :p - n] = 0
        L[n, p + n + 1:] = 0
        for m in range(1, n + 1):
            L[n, p - m] = (-1) ** m * np.conj(L[n, p + m])
        L[n, p] = L[n, p].real
    cp = np.array([0.5, 0.5])
    cc = cp + np.array([0.05, -0.05])
    Lc = (ops.l2l((cc[0] - cp[0], cc[1] - cp[1], 0.0)) @ L.ravel()).reshape(L.shape)
    tg = cc + g.uniform(-0.05, 0.05, size=(40, 2))
    a = fmm.evaluate_local(p, L, cp, tg)
    b = fmm.evaluate_local(p, Lc, cc, tg)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
    assert np.max(np.abs(a.imag)) < 1e-13 * np.max(np.abs(a))


def test_m2l_then_l2p_matches_direct_within_bound():
    g = np.random.default_rng(2)
    c = 0.03
    h = 0.1
    zs = np.array([0.2, 0.2])
    zt = zs + np.array([2 * h, 1 * h])           # a V-list offset
    src = zs + g.uniform(-h / 2, h / 2, size=(50, 2))
    tgt = zt + g.uniform(-h / 2, h / 2, size=(50, 2))
    u = g.uniform(-1, 1, 50)
    exact = np.array([np.sum(u / np.sqrt(np.sum((t - src) ** 2, axis=1) + c * c)) for t in tgt])
    errs = []
    for p in (4, 8, 12, 16):
        ops = fmm.ops_for(p)
        M = fmm.multipole_of_points(p, zs, src, u)
        L = (ops.m2l((zt[0] - zs[0], zt[1] - zs[1], c)) @ M.ravel()).reshape(M.shape)
        val = fmm.evaluate_local(p, L, zt, tgt)
        errs.append(np.max(np.abs(val - exact)))
        # FMM bound with both radii: sum|u| (rs+rt)^{p+1} / ((|d|-rs-rt) |d|^{p+1})
        rs = rt = h / math.sqrt(2)
        d = math.sqrt(np.sum((zt - zs) ** 2) + c * c)
        r = (rs + rt) / d
        assert errs[-1] <= np.sum(np.abs(u)) * r ** (p + 1) / ((1 - r) * d)
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_fmm_invariants_and_convergence():
    pts = W.clustered_points(300, 8, 1200, 0.03, 3)
    u = W.random_vector(pts.shape[0], 3)
    c = 0.01
    bd = dense.matvec(pts, c, u)
    prev = None
    for p in (4, 8, 12):
        out, st = fmm.fmm_matvec(pts, c, u, p, 16, return_state=True)
        assert np.max(np.abs(out.imag)) < 1e-12 * np.max(np.abs(bd))
        assert np.max(np.abs(st["M"][:, fmm.odd_mask(p)])) < 1e-13 * np.max(np.abs(st["M"]))
        err = np.linalg.norm(out.real - bd) / np.linalg.norm(bd)
        if prev is not None:
            assert err < prev / 5
        prev = err
    assert prev < 1e-6


def test_fmm_uniform_small_c():
    pts = W.uniform_points(2000, 1)
    u = W.random_vector(2000, 1)
    b = fmm.fmm_matvec(pts, 0.1, u, 10, 32)
    bd = dense.matvec(pts, 0.1, u)
    assert np.linalg.norm(b - bd) / np.linalg.norm(bd) < 1e-6


def test_planted_m2l_sign_error_is_caught(monkeypatch):
    # a dropped (-1)^k in M2L must break the convergence pin
    orig = fmm._Ops.m2l

    def bad(self, d):
        T_ = orig(self, d).copy()
        return np.abs(T_.real) + 1j * T_.imag
    monkeypatch.setattr(fmm._Ops, "m2l", bad)
    pts = W.uniform_points(800, 2)
    u = W.random_vector(800, 2)
    b = fmm.fmm_matvec(pts, 0.05, u, 8, 16)
    bd = dense.matvec(pts, 0.05, u)
    assert np.linalg.norm(b - bd) / np.linalg.norm(bd) > 1e-3


# ----------------------------------------------------------------- Algorithm 1

def test_treecode_covers_every_pair_once():
    pts = W.halton_points(2000)
    u = W.random_vector(2000, 6)
    for L in (1, 2, 3):
        _, far, near = treecode.treecode_matvec(pts, 1.0, u, 4, L, count_pairs=True)
        assert far + near == 2000 * 2000


def test_treecode_error_within_theorem_2_1_and_table_1():
    n = 4000
    pts = W.halton_points(n)
    u = W.random_vector(n, 6)
    bd = dense.matvec(pts, 1.0, u)
    # at level 1 with t = 1 every far pair has ratio <= sqrt(2/73) (worked example),
    # so |b_i - (A u)_i| <= sum_j |u_j| * bound
    r = math.sqrt(2.0 / 73.0)
    pair_bound = r ** 11 / ((1 - r) * math.sqrt(73) / 8)
    rows = golden("table1.txt")
    e_table = min(float(row[3]) for row in rows)
    for L in (1, 2):
        b = treecode.treecode_matvec(pts, 1.0, u, 10, L)
        assert np.max(np.abs(b - bd)) <= np.sum(np.abs(u)) * pair_bound
        einf = np.max(np.abs(b - bd)) / np.max(np.abs(bd))
        assert einf < e_table                 # at least as accurate as Table 1 reports
    b20 = treecode.treecode_matvec(pts, 1.0, u, 20, 1)
    assert np.max(np.abs(b20 - bd)) / np.max(np.abs(bd)) < 1e-13


def test_treecode_planted_index_error_is_caught(monkeypatch):
    # a wrong packed index k (colliding terms) must break the accuracy pin
    monkeypatch.setattr(treecode, "packed_index", lambda n, m: n * (n + 1) // 2 + max(m - 1, 0))
    pts = W.halton_points(1500)
    u = W.random_vector(1500, 6)
    bd = dense.matvec(pts, 1.0, u)
    b = treecode.treecode_matvec(pts, 1.0, u, 10, 1)
    assert np.max(np.abs(b - bd)) / np.max(np.abs(bd)) > 1e-6
