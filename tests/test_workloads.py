"""The seeded synthetic inputs follow their stated recipes (no GPU).

The generators hold none of the method's arithmetic; these checks pin them to
the configurations they stand for: sizes, parameters, value ranges, the
Halton sequence's definition and the nearest-neighbour spacing's.
"""
import math

import numpy as np
import pytest

from paper_2205_04194_gb300 import workloads as W


def test_halton_points_are_radical_inverses_in_bases_2_and_3():
    h = W.halton_points(6)
    expect = [[1 / 2, 1 / 3], [1 / 4, 2 / 3], [3 / 4, 1 / 9], [1 / 8, 4 / 9], [5 / 8, 7 / 9], [3 / 8, 2 / 9]]
    assert np.allclose(h, expect, rtol=0, atol=1e-15)
    assert np.array_equal(W.halton_points(3, start=4), W.halton_points(6)[3:])


def test_mean_nn_spacing_on_a_grid_is_the_grid_step():
    g = np.stack(np.meshgrid(np.arange(7) * 0.125, np.arange(5) * 0.125), axis=-1).reshape(-1, 2)
    assert W.mean_nn_spacing(g) == pytest.approx(0.125, rel=1e-15)


def test_clustered_1m_recipe():
    wl = W.clustered_1m()
    assert wl.n == 1_000_000 and wl.c == 0.01 and wl.leaf == 64 and wl.domain == (0.0, 0.0, 1.0)
    assert wl.points.min() >= 0.0 and wl.points.max() <= 1.0
    cl = wl.points[:700_000].reshape(8, 87_500, 2)
    centres = np.median(cl, axis=1)
    assert np.all((centres > 0.1 - 0.01) & (centres < 0.9 + 0.01))     # centres in [0.1, 0.9]^2
    spread = np.std(cl - centres[:, None, :], axis=1)
    assert np.all(np.abs(spread - 0.03) < 0.002)                        # sigma 0.03 (clamping aside)
    assert np.all(np.abs(wl.v) <= 1.0)


def test_uniform_100k_shape_is_twice_the_mean_nn_spacing():
    wl = W.uniform_100k()
    h = W.mean_nn_spacing(wl.points)
    assert wl.c == pytest.approx(2.0 * h)
    # Poisson process of intensity N: mean nearest-neighbour distance 1 / (2 sqrt(N))
    assert h == pytest.approx(0.5 / math.sqrt(wl.n), rel=0.03)
    assert wl.p == 12 and wl.leaf == 64


def test_batched_256_recipe():
    probs = W.batched_256()
    assert len(probs) == 256
    ns = np.array([x.shape[0] for x, _, _ in probs])
    cs = np.array([c for _, c, _ in probs])
    assert ns.min() >= 1000 and ns.max() <= 50_000
    assert np.median(ns) == pytest.approx(math.sqrt(1e3 * 5e4), rel=0.25)   # log-uniform
    assert cs.min() >= 0.01 and cs.max() <= 0.2
    for x, _, r in probs[:4]:
        assert r.shape == (4, x.shape[0]) and np.allclose(r[0], W.franke(x))


def test_grad_200k_and_plain_2k_recipes():
    g = W.grad_200k()
    assert g["train"].shape == (200_000, 2) and g["val"].shape == (20_000, 2) and g["c"] == 0.05
    assert np.allclose(g["f"], np.exp(-10 * ((g["train"][:, 0] - 0.5) ** 2 + (g["train"][:, 1] - 0.5) ** 2)))
    p = W.plain_2k()
    assert p.n == 2000 and p.c == 0.1 and p.p == 10 and p.leaf == 32


def test_inputs_are_reproducible_from_their_seeds():
    assert np.array_equal(W.uniform_points(100, 9), W.uniform_points(100, 9))
    assert not np.array_equal(W.uniform_points(100, 9), W.uniform_points(100, 9, stream=1))
    assert np.array_equal(W.random_vector(50, 3, nrhs=2), W.random_vector(50, 3, nrhs=2))
