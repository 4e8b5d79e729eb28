"""Pins for oracle.harmonics: Section 2.1 of the paper (Eqs. (6)-(9), Theorem 2.1)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from conftest import golden
from oracle import harmonics as H


def test_legendre_poly_matches_numpy_series():
    x = np.linspace(-1, 1, 101)
    for n in range(0, 25):
        c = np.zeros(n + 1)
        c[n] = 1.0
        assert np.allclose(H.legendre_poly(n, x), npleg.legval(x, c), atol=1e-13)
        assert np.allclose(H.legendre_table(n, x)[..., n, 0], npleg.legval(x, c), atol=1e-12)


def test_legendre_closed_forms():
    # P_n^m(0) = (-1)^{(n-m)/2} (n+m)! / (2^n ((n-m)/2)! ((n+m)/2)!) for n+m even, else 0
    P0 = H.legendre_table(20, 0.0)
    for n in range(21):
        for m in range(n + 1):
            if (n + m) % 2:
                want = 0.0
            else:
                want = ((-1) ** ((n - m) // 2) * math.factorial(n + m)
                        / (2 ** n * math.factorial((n - m) // 2) * math.factorial((n + m) // 2)))
            assert P0[n, m] == pytest.approx(want, rel=1e-12, abs=1e-300)
    # P_n^m(1) = delta_{m0}; P_m^m(x) = (2m-1)!! (1-x^2)^{m/2}
    P1 = H.legendre_table(15, 1.0)
    assert np.allclose(P1[:, 0], 1.0) and np.allclose(np.tril(P1, -1)[:, 1:], 0.0)
    x = 0.3
    Px = H.legendre_table(12, x)
    for m in range(13):
        dfact = float(np.prod(np.arange(1, 2 * m, 2))) if m else 1.0
        assert Px[m, m] == pytest.approx(dfact * (1 - x * x) ** (m / 2), rel=1e-13)


def test_legendre_bounded_by_one():
    # |P_n(x)| <= 1 on [-1, 1] (used in the proof of Theorem 2.1)
    x = np.linspace(-1, 1, 2001)
    for n in range(40):
        assert np.max(np.abs(H.legendre_poly(n, x))) <= 1.0 + 1e-12


def _unit(th, om):
    return np.array([np.sin(th) * np.cos(om), np.sin(th) * np.sin(om), np.cos(th)])


def test_addition_theorem_against_direct_angle():
    # P_n(cos alpha) = sum_m eps_m (n-m)!/(n+m)! P_n^m(cos th_y) P_n^m(cos th_x) cos(m dom)
    g = np.random.default_rng(0)
    for _ in range(50):
        tx, ty = g.uniform(0, np.pi, 2)
        ox, oy = g.uniform(-np.pi, np.pi, 2)
        cosa = float(_unit(tx, ox) @ _unit(ty, oy))
        for n in range(0, 18):
            assert H.addition_theorem_sum(n, tx, ty, ox, oy) == pytest.approx(
                float(H.legendre_poly(n, cosa)), abs=1e-12)


def test_truncated_series_obeys_theorem_2_1():
    g = np.random.default_rng(1)
    X = g.normal(size=(400, 3))
    Y = g.normal(size=(400, 3))
    rx = np.linalg.norm(X, axis=1)
    ry = np.linalg.norm(Y, axis=1)
    keep = np.abs(rx - ry) / np.maximum(rx, ry) > 0.15
    X, Y = X[keep], Y[keep]
    exact = 1.0 / np.linalg.norm(X - Y, axis=1)
    prev = None
    for M in (2, 5, 10, 20):
        err = np.abs(exact - H.truncated_series(X, Y, M))
        bound = H.thm21_bound(np.linalg.norm(X, axis=1), np.linalg.norm(Y, axis=1), M)
        assert np.all(err <= bound * (1 + 1e-9) + 8 * np.finfo(float).eps * exact)
        if prev is not None:
            assert np.median(err) < np.median(prev)
        prev = err


@pytest.mark.parametrize("case", ["a", "b"])
def test_figure1_setup(case):
    rows = {r[0]: r[1:] for r in golden("fig1_setup.txt")}
    ry = float(rows["rho_y"][0])
    rxs = np.linspace(float(rows["rho_x_min"][0]), float(rows["rho_x_max"][0]), 200)
    if case == "a":
        tx = ty = ox = oy = np.pi / 3
    else:
        tx, ty, ox, oy = np.pi, np.pi / 4, np.pi / 3, np.pi / 2
    Y = ry * _unit(ty, oy)
    errs = {}
    for M in [int(v) for v in rows["M"]]:
        X = rxs[:, None] * _unit(tx, ox)[None, :]
        exact = 1.0 / np.linalg.norm(X - Y[None, :], axis=1)
        err = np.abs(exact - H.truncated_series(X, np.broadcast_to(Y, X.shape), M))
        assert np.all(err <= H.thm21_bound(rxs, ry, M) * (1 + 1e-9) + 8 * np.finfo(float).eps * exact)
        errs[M] = err
    # pointwise the tail can change sign with M, but over the rho_x range a
    # larger M does better (the trend Figure 1 shows)
    for lo, hi in ((5, 10), (10, 20)):
        assert np.median(errs[hi]) < np.median(errs[lo])
        assert np.max(errs[hi][rxs > 2.0]) < np.max(errs[lo][rxs > 2.0])
    # error is large when rho_x ~ rho_y and tiny far away
    assert errs[10][0] > 1e-3 * errs[10][0] + errs[10][-1]


def test_worked_example_bound():
    rows = {r[0]: float(r[1]) for r in golden("worked_example.txt")}
    rho_y = math.sqrt(rows["rho_y_max_sq_times_64"]) / 8
    rho_x = math.sqrt(rows["rho_x_min_sq_times_64"]) / 8
    assert rho_y / rho_x == pytest.approx(rows["ratio"], abs=5e-5)
    # the printed bound uses the rounded ratio 0.1655 and 1/rho_x with rho_x = sqrt(73)/8
    for M, key in ((10, "bound_M10"), (20, "bound_M20")):
        r = rows["ratio"]
        b = r ** (M + 1) / ((1 - r) * rho_x)
        assert b == pytest.approx(rows[key], rel=5e-3)


def test_worked_example_empirical_error_below_bound():
    # every level-1 well-separated (source block, target point) pair at t = 1
    t = 1.0
    g = np.random.default_rng(2)
    h = 0.25
    worst = 0.0
    for bx in range(4):
        for by in range(4):
            z = np.array([(bx + 0.5) * h, (by + 0.5) * h])
            src = z + g.uniform(-h / 2, h / 2, size=(60, 2))
            src = np.concatenate([src, z + np.array([[h / 2, h / 2], [-h / 2, h / 2]])])
            for qx in range(4):
                for qy in range(4):
                    if max(abs(qx - bx), abs(qy - by)) <= 1:
                        continue
                    tgt = np.array([qx * h, qy * h]) + g.uniform(0, h, size=(30, 2))
                    Xv = np.concatenate([tgt - z, np.full((tgt.shape[0], 1), t)], axis=1)
                    Yv = np.concatenate([src - z, np.zeros((src.shape[0], 1))], axis=1)
                    XX = np.repeat(Xv, Yv.shape[0], axis=0)
                    YY = np.tile(Yv, (Xv.shape[0], 1))
                    exact = 1.0 / np.linalg.norm(XX - YY, axis=1)
                    worst = max(worst, float(np.max(np.abs(exact - H.truncated_series(XX, YY, 10)))))
    r = math.sqrt(2.0 / 73.0)
    assert worst < r ** 11 / ((1 - r) * math.sqrt(73) / 8)


def test_solid_harmonics_reproduce_eq7_degree_by_degree():
    # sum_{m=-n}^{n} conj(U_n^m(Y)) T_n^m(X) equals the degree-n term of Eq. (7)
    g = np.random.default_rng(3)
    p = 12
    for _ in range(20):
        X = g.normal(size=3) * 2
        Y = g.normal(size=3) * 0.5
        U = H.regular(p, Y)
        T = H.irregular(p, X)
        rx, tx, ox = H.spherical(X)
        ry, ty, oy = H.spherical(Y)
        for n in range(p + 1):
            lhs = np.sum(np.conj(U[n]) * T[n])
            rhs = H.addition_theorem_sum(n, tx, ty, ox, oy) * ry ** n / rx ** (n + 1)
            assert abs(lhs.imag) < 1e-12 * (1 + abs(rhs))
            assert lhs.real == pytest.approx(float(rhs), rel=1e-10, abs=1e-14)


def test_regular_harmonic_on_axis_and_addition():
    z = 0.7
    U = H.regular(10, np.array([0.0, 0.0, z]))
    for n in range(11):
        assert U[n, 10].real == pytest.approx(z ** n / math.factorial(n), rel=1e-13)
        assert np.allclose(np.delete(U[n], 10), 0.0)
    g = np.random.default_rng(4)
    p = 8
    for _ in range(5):
        a, b = g.normal(size=3), g.normal(size=3)
        Ua, Ub, Uab = H.regular(p, a), H.regular(p, b), H.regular(p, a + b)
        for n in range(p + 1):
            for m in range(-n, n + 1):
                s = 0j
                for k in range(n + 1):
                    for l in range(-k, k + 1):
                        if abs(m - l) <= n - k:
                            s += Ua[k, l + p] * Ub[n - k, m - l + p]
                assert abs(s - Uab[n, m + p]) < 1e-12 * (1 + abs(Uab[n, m + p]))


def test_irregular_translation():
    g = np.random.default_rng(5)
    P, q = 36, 5
    for _ in range(3):
        x = g.normal(size=3) * 3
        y = g.normal(size=3) * 0.25
        Tx, Uy, Txy = H.irregular(P, x), H.regular(P, y), H.irregular(q, x - y)
        for n in range(q + 1):
            for m in range(-n, n + 1):
                s = 0j
                for k in range(P - n + 1):
                    for l in range(-k, k + 1):
                        s += np.conj(Uy[k, l + P]) * Tx[n + k, m + l + P]
                assert abs(s - Txy[n, m + q]) < 1e-10 * abs(Txy[0, q])


def test_laplace_pair_equals_green_function():
    g = np.random.default_rng(6)
    X = g.normal(size=(100, 3)) * 3
    Y = g.normal(size=(100, 3)) * 0.5
    ok = np.linalg.norm(Y, axis=1) < 0.6 * np.linalg.norm(X, axis=1)
    X, Y = X[ok], Y[ok]
    exact = 1.0 / np.linalg.norm(X - Y, axis=1)
    for p in (4, 8, 16):
        err = np.abs(H.laplace_pair(p, X, Y) - exact)
        assert np.all(err <= H.thm21_bound(np.linalg.norm(X, axis=1), np.linalg.norm(Y, axis=1), p)
                      * (1 + 1e-9) + 16 * np.finfo(float).eps * exact)
