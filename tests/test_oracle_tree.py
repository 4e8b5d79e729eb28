"""Pins for oracle.tree (O4): the partition of Section 2.2 and its interaction sets."""
import numpy as np
import pytest

from oracle import tree as T
from paper_2205_04194_gb300 import workloads as W


def test_interleave_known_values():
    assert T.interleave(np.array([1]), np.array([0]))[0] == 1
    assert T.interleave(np.array([0]), np.array([1]))[0] == 2
    assert T.interleave(np.array([0xFFFF]), np.array([0]))[0] == 0x55555555
    assert T.interleave(np.array([0]), np.array([0xFFFF]))[0] == 0xAAAAAAAA
    assert T.interleave(np.array([0x8000]), np.array([0x8000]))[0] == 0xC0000000
    g = np.random.default_rng(0)
    qx = g.integers(0, 65536, 1000).astype(np.uint32)
    qy = g.integers(0, 65536, 1000).astype(np.uint32)
    rx, ry = T.deinterleave(T.interleave(qx, qy))
    assert np.array_equal(rx, qx) and np.array_equal(ry, qy)


def test_quantisation_edges():
    dom = (0.0, 0.0, 1.0)
    pts = np.array([[0.0, 0.0], [1.0, 1.0], [0.5, 0.25], [-0.1, 1.5], [np.nextafter(0.5, 0), 0.75]])
    qx, qy = T.quantise(pts, dom)
    assert list(qx) == [0, 65535, 32768, 0, 32767]
    assert list(qy) == [0, 65535, 16384, 65535, 49152]


def test_default_domain():
    pts = np.array([[2.0, 3.0], [2.5, 3.1], [2.2, 4.0]])
    assert T.default_domain(pts) == (2.0, 3.0, 1.0)
    assert T.default_domain(np.array([[1.0, 1.0]])) == (1.0, 1.0, 1.0)


def test_stable_sort_keeps_input_order_of_ties():
    pts = np.array([[0.1, 0.1], [0.9, 0.9], [0.1, 0.1], [0.1, 0.1]])
    t = T.build_tree(pts, 1, (0.0, 0.0, 1.0))
    assert list(t.perm) == [0, 2, 3, 1]
    # identical points cannot be separated: they end in one leaf at level 16
    leaf_of_dups = [b for b in range(t.nbox) if t.is_leaf[b] and t.end[b] - t.begin[b] == 3]
    assert len(leaf_of_dups) == 1 and t.level[leaf_of_dups[0]] == T.MAX_LEVEL


def _mixed(seed, n):
    g = np.random.default_rng(seed)
    return np.concatenate([g.random((n // 2, 2)), 0.3 + 0.01 * g.standard_normal((n - n // 2, 2))])


@pytest.mark.parametrize("seed,n,leaf", [(0, 200, 4), (1, 300, 3), (2, 150, 1), (3, 257, 8), (4, 64, 2)])
def test_lists_match_set_definitions_and_cover_every_pair_once(seed, n, leaf):
    t = T.build_tree(_mixed(seed, n), leaf)
    bf = T.brute_force_lists(t)
    for k in "UVWX":
        assert bf[k] == getattr(t, k), k
    cov = T.coverage(t)
    assert cov.min() == 1 and cov.max() == 1


def test_box_rules():
    pts = W.clustered_points(1200, 8, 4000, 0.03, 3)
    t = T.build_tree(pts, 16)
    cnt = t.end - t.begin
    assert np.all(cnt[~t.is_leaf] > 16)
    assert np.all((cnt[t.is_leaf] <= 16) | (t.level[t.is_leaf] == T.MAX_LEVEL))
    assert np.all(cnt > 0)
    # (level, prefix) order and children contiguous inside their parent
    key = t.level.astype(np.int64) * (1 << 32) + t.prefix.astype(np.int64)
    assert np.all(np.diff(key) > 0)
    for b in range(t.nbox):
        ch = t.children(b)
        if ch:
            assert t.begin[ch[0]] == t.begin[b] and t.end[ch[-1]] == t.end[b]
            for a, c in zip(ch[:-1], ch[1:]):
                assert t.end[a] == t.begin[c]
    # codes sorted, perm a permutation
    assert np.all(np.diff(t.sorted_codes.astype(np.int64)) >= 0)
    assert np.array_equal(np.sort(t.perm), np.arange(pts.shape[0]))


def test_uniform_tree_counts_of_the_paper():
    # 4^5 points on a regular grid, leaf 1: a uniform tree of depth 5.
    g = (np.arange(32) + 0.5) / 32
    pts = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    t = T.build_tree(pts, 1, (0.0, 0.0, 1.0))
    assert int(t.level.max()) == 5 and np.all(t.level[t.is_leaf] == 5)
    vl = np.array([len(v) for v in t.V])
    assert vl[t.level == 2].max() == 12          # first level (4x4): at most 12 well-separated blocks
    assert vl[t.level >= 3].max() == 27          # finer levels: at most 27
    ul = np.array([len(u) for u in t.U])
    assert ul[t.is_leaf].max() == 9              # at most 9 not-well-separated blocks
    assert all(len(w) == 0 for w in t.W) and all(len(x) == 0 for x in t.X)
