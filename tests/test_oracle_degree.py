"""Pins of the expected-average-degree formula and the search for c (App. B.2).

* f(c) against a brute-force sum over ordered pairs of E[X_uv], each computed
  by numerical integration over the L_inf torus distance, whose law is
  P(r <= t) = (2t)^d for t <= 1/2 -- no closed form shared with the oracle.
* f(c) against the Monte-Carlo mean degree of the all-pairs sampler.
* The search inverts f.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def _ex_uv(c, q, d, T):
    dens = lambda r: d * 2.0 ** d * r ** (d - 1)  # noqa: E731
    if T == 0.0:
        t = c * q ** (1.0 / d)
        return min(1.0, (2.0 * t) ** d)
    kink = (c ** T * q) ** (1.0 / d)  # p = 1 below the kink
    if kink >= 0.5:
        return 1.0
    short = (2.0 * kink) ** d
    f = lambda r: c * (q / r ** d) ** (1.0 / T) * dens(r)  # noqa: E731
    long_, _ = integrate.quad(f, kink, 0.5, epsabs=0, epsrel=1e-12, limit=200)
    return short + long_


def _brute_force_degree(c, w, d, T):
    W = math.fsum(w)
    n = len(w)
    tot = 0.0
    for u in range(n):
        for v in range(n):
            if u != v:
                tot += _ex_uv(c, w[u] * w[v] / W, d, T)
    return tot / n


@pytest.mark.parametrize("d,T", [(1, 0.0), (2, 0.0), (1, 0.5), (2, 0.3), (3, 0.7), (4, 0.9)])
def test_degree_formula_matches_integration(d, T):
    rng = np.random.default_rng(100 + d)
    w = 1.0 + rng.pareto(1.3, 25)
    W = O.exact_sum(w)
    for c in (0.01, 0.5, 4.0, 40.0):
        ref = _brute_force_degree(c, w, d, T)
        got = O.girg_avg_degree(c, w, d, T, W)
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-12), (c, got, ref)


@pytest.mark.parametrize("d,T", [(1, 0.5), (2, 0.0), (2, 0.7)])
def test_degree_formula_matches_monte_carlo(d, T):
    n, runs = 300, 200
    w, _ = O.girg_points(n, d, 2.5, 1.0, 5)
    W = O.exact_sum(w)
    c = O.girg_solve_c(6.0, w, d, T, W)
    degs = []
    for s in range(runs):
        _, X = O.girg_points(n, d, 2.5, 1.0, 1000 + s)  # fresh positions, same weights
        e = O.girg_allpairs(X, w, W, T, c, 77 + s)
        degs.append(2.0 * len(e) / n)
    degs = np.array(degs)
    se = degs.std(ddof=1) / math.sqrt(runs)
    assert abs(degs.mean() - 6.0) < 4.5 * se + 1e-9


@pytest.mark.parametrize("d,T,target", [(1, 0.5, 10.0), (2, 0.5, 10.0), (3, 0.7, 16.0),
                                        (2, 0.0, 16.0), (4, 0.0, 16.0)])
def test_solver_inverts_degree(d, T, target):
    w, _ = O.girg_points(20000, d, 2.2, 1.0, 9)
    W = O.exact_sum(w)
    c = O.girg_solve_c(target, w, d, T, W)
    assert c > 0
    assert O.girg_avg_degree(c, w, d, T, W) == pytest.approx(target, rel=1e-10)
