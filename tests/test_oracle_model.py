"""Pins of the oracle's model formulas and input distributions.

* Eq. 1 and the threshold variant against values worked out by hand and by
  mpmath, including the inclusive tie of the threshold case (Sec. 2.1).
* The HRG distance and connection probability against mpmath evaluations of
  the textbook formulas of Sec. 2.2 at 60 digits.
* Weights, positions and HRG radii against their distributions (KS tests).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

mp = pytest.importorskip("mpmath")


def test_girg_p_hand_values():
    # d = 1, T = 1/2: p = c (q / r)^2, q = w_u w_v / W
    W, wu, wv = 100.0, 2.0, 5.0  # q = 0.1
    assert O.girg_p(1, 0.5, 0.5, W, wu, wv, 2 ** 29) == pytest.approx(0.5 * (0.1 / 0.125) ** 2,
                                                                        rel=1e-15)
    # capped at 1 (Eq. 1 min)
    assert O.girg_p(1, 0.5, 2.0, W, wu, wv, 2 ** 29) == 1.0
    # d = 2, r = 1/2: p = c (q / r^2)^(1/T)
    assert O.girg_p(2, 0.5, 0.5, W, wu, wv, 2 ** 31) == pytest.approx(0.5 * 0.4 ** 2, rel=1e-15)
    # coincident points: r = 0 gives p = 1
    assert O.girg_p(3, 0.7, 1e-9, W, wu, wv, 0) == 1.0
    # non-integer 1/T against mpmath: c outside the power, q / r^d inside (Eq. 1)
    mp.mp.dps = 40
    rng = np.random.default_rng(3)
    for _ in range(500):
        d = int(rng.integers(1, 5))
        T = float(rng.uniform(0.05, 0.95))
        c = float(np.exp(rng.uniform(-5, 5)))
        W = float(np.exp(rng.uniform(5, 20)))
        wu, wv = (float(np.exp(rng.uniform(0, 8))) for _ in range(2))
        D = int(rng.integers(1, 2 ** 31))
        r = mp.mpf(D) / 2 ** 32
        ref = mp.mpf(c) * mp.power((mp.mpf(wu) * wv / W) / r ** d, 1 / mp.mpf(T))
        ref = min(ref, mp.mpf(1))
        got = O.girg_p(d, T, c, W, wu, wv, D)
        assert abs(got - ref) <= 1e-12 * ref + 1e-300


def test_girg_threshold_inclusive_tie():
    # d = 1: threshold c q = 0.25 with c = 1, q = 0.25 -> r = 2^30 / 2^32 is an edge
    W, wu, wv = 100.0, 5.0, 5.0
    assert O.girg_thresh_edge(1, 1.0, W, wu, wv, 2 ** 30)
    assert not O.girg_thresh_edge(1, 1.0, W, wu, wv, 2 ** 30 + 1)
    # d = 2: threshold c q^(1/2) = 0.5
    assert O.girg_thresh_edge(2, 1.0, W, wu, wv, 2 ** 31)
    assert not O.girg_thresh_edge(2, 0.999, W, wu, wv, 2 ** 31)


def _mp_coshd(ru, rv, D):
    dt = 2 * mp.pi * mp.mpf(D) / 2 ** 32
    ru, rv = mp.mpf(ru), mp.mpf(rv)
    return mp.cosh(ru) * mp.cosh(rv) - mp.sinh(ru) * mp.sinh(rv) * mp.cos(dt)


def test_hrg_coshd_against_mpmath():
    """Sec. 2.2 distance, evaluated naively at 60 digits, vs the stable FP64 form."""
    mp.mp.dps = 60
    rng = np.random.default_rng(4)
    for _ in range(3000):
        ru = float(rng.uniform(0, 35))
        rv = ru + float(rng.normal(0, 0.5)) if rng.random() < 0.5 else float(rng.uniform(0, 35))
        rv = abs(rv)
        D = int(rng.integers(0, 2 ** 31)) if rng.random() < 0.5 else int(rng.integers(0, 2 ** 12))
        ref = _mp_coshd(ru, rv, D)
        got = O.hrg_coshd(ru, rv, D)
        assert abs(got - ref) / ref < 1e-14, (ru, rv, D)


def test_hrg_p_against_mpmath():
    mp.mp.dps = 60
    rng = np.random.default_rng(5)
    for _ in range(1500):
        R = float(rng.uniform(10, 40))
        T = float(rng.uniform(0.05, 0.95))
        ru, rv = float(rng.uniform(R / 2, R)), float(rng.uniform(R / 2, R))
        D = int(rng.integers(0, 2 ** 31))
        dist = mp.acosh(_mp_coshd(ru, rv, D))
        ref = 1 / (mp.exp((dist - R) / (2 * T)) + 1)
        got = O.hrg_p(T, R, ru, rv, D)
        assert abs(got - ref) <= 1e-12 * ref + 1e-300
    # threshold: edge iff d < R (strict)
    R = 20.0
    assert O.hrg_p(0.0, R, 5.0, 5.0, 0) == 1.0
    assert O.hrg_p(0.0, R, 19.9, 19.9, 2 ** 31) == 0.0


def test_weights_are_pareto():
    n, beta = 200_000, 2.5
    w, X = O.girg_points(n, 3, beta, 1.0, 11)
    assert w.min() >= 1.0
    res = stats.kstest(w, lambda x: 1.0 - np.power(x, -(beta - 1.0)))
    assert res.pvalue > 1e-3
    # w_min scales the distribution
    w2, _ = O.girg_points(1000, 1, beta, 3.0, 11)
    assert np.array_equal(w2, 3.0 * w[:1000])


def test_positions_are_uniform_and_independent_of_d():
    n = 100_000
    _, X3 = O.girg_points(n, 3, 2.5, 1.0, 12)
    _, X5 = O.girg_points(n, 5, 2.5, 1.0, 12)
    assert np.array_equal(X3, X5[:, :3])
    for k in range(5):
        res = stats.kstest(X5[:, k] / 2.0 ** 32, "uniform")
        assert res.pvalue > 1e-3
    assert abs(np.corrcoef(X5[:, 0].astype(float), X5[:, 4].astype(float))[0, 1]) < 0.02


def test_hrg_radii_follow_density():
    """f(r) = alpha sinh(alpha r) / (cosh(alpha R) - 1) on [0, R) (Sec. 2.2)."""
    n, alpha, R = 200_000, 0.75, 25.0
    r, X = O.hrg_points(n, alpha, R, 13)
    assert r.min() >= 0.0 and r.max() <= R
    res = stats.kstest(r, lambda x: (np.cosh(alpha * x) - 1.0) / (np.cosh(alpha * R) - 1.0))
    assert res.pvalue > 1e-3
    assert stats.kstest(X / 2.0 ** 32, "uniform").pvalue > 1e-3
    # HRG -> GIRG mapping (Sec. 2.3): w = e^((R - r) / 2) >= 1
    for rv in (0.0, 3.0, R):
        assert O.hrg_weight(rv, R) == pytest.approx(math.exp((R - rv) / 2), rel=1e-15)
