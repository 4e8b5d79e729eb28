"""GPU tree build vs the oracle: Morton codes, permutation, boxes and U/V/W/X lists, bit-exact."""
import numpy as np
import pytest

from gpu_util import cuda, need_gpu
from oracle import tree as T
from paper_2205_04194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _compare(pts, leaf, domain=None, c=0.05, p=6):
    need_gpu()
    from paper_2205_04194_gb300 import imq
    plan = imq.Plan(cuda(pts), c, p, leaf, domain=domain)
    g = plan.export_tree()
    o = T.build_tree(pts, leaf, domain)
    info = plan.info()
    if domain is None:
        assert (info["x0"], info["y0"], info["side"]) == o.domain
    assert np.array_equal(g["codes"], o.sorted_codes)
    assert np.array_equal(g["perm"], o.perm)
    assert info["n_boxes"] == o.nbox
    assert np.array_equal(g["level"], o.level)
    assert np.array_equal(g["prefix"], o.prefix)
    assert np.array_equal(g["begin"], o.begin) and np.array_equal(g["end"], o.end)
    assert np.array_equal(g["parent"], o.parent)
    assert np.array_equal(g["child"], o.child)
    for name in "UVWX":
        off, items = plan.export_list(name)
        ooff, oitems = o.csr(name)
        assert np.array_equal(off, ooff), name
        assert np.array_equal(items, oitems), name
    plan.close()
    return o


def test_tree_uniform_2k():
    _compare(W.uniform_points(2000, 1), 32, (0.0, 0.0, 1.0))


def test_tree_clustered_default_domain():
    pts = W.clustered_points(2500, 8, 10000, 0.03, 3)
    o = _compare(pts, 64)
    assert len(o.W) and sum(len(w) for w in o.W) > 0       # adaptive lists are exercised


def test_tree_tiny_and_leaf_one():
    _compare(np.array([[0.3, 0.7]]), 4)
    _compare(W.uniform_points(5, 2), 1)
    _compare(W.uniform_points(70, 3), 1, (0.0, 0.0, 1.0))


def test_tree_duplicates_reach_max_level():
    pts = np.concatenate([W.uniform_points(300, 4), np.repeat([[0.25, 0.5]], 5, axis=0)])
    o = _compare(pts, 2)
    assert o.level.max() == T.MAX_LEVEL


def test_duplicate_points_rejected_on_request():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts = np.concatenate([W.uniform_points(100, 5), [[0.5, 0.5], [0.5, 0.5]]])
    with pytest.raises(imq.ImqError) as e:
        imq.Plan(cuda(pts), 0.1, 6, 8, check_duplicates=True)
    assert e.value.status == 2


def test_nonfinite_rejected():
    need_gpu()
    from paper_2205_04194_gb300 import imq
    pts = W.uniform_points(50, 6)
    pts[7, 1] = np.nan
    with pytest.raises(imq.ImqError) as e:
        imq.Plan(cuda(pts), 0.1, 6, 8)
    assert e.value.status == 1


def test_tree_full_size_clustered_1m():
    wl = W.clustered_1m()
    _compare(wl.points, wl.leaf, wl.domain, c=wl.c, p=8)
