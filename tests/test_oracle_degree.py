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


def _ex_uv(K, q, d, T):
    """E[X_uv] for p = min{1, (K q / r^d)^(1/T)} (Eq. 1 with K = c^T; T = 0: r^d <= K q)."""
    dens = lambda r: d * 2.0 ** d * r ** (d - 1)  # noqa: E731
    kink = (K * q) ** (1.0 / d)  # p = 1 below the kink
    if T == 0.0:
        return min(1.0, (2.0 * kink) ** d)
    if kink >= 0.5:
        return 1.0
    short = (2.0 * kink) ** d
    # beyond the kink, in r = kink e^s (smooth even when 1/T is large)
    f = lambda s: (math.exp((math.log(K * q) - d * math.log(kink) - d * s) / T)  # noqa: E731
                   * dens(kink * math.exp(s)) * kink * math.exp(s))
    long_, _ = integrate.quad(f, 0.0, math.log(0.5 / kink), epsabs=0, epsrel=1e-12, limit=200)
    return short + long_


def _brute_force_degree(K, w, d, T):
    W = math.fsum(w)
    n = len(w)
    tot = 0.0
    for u in range(n):
        for v in range(n):
            if u != v:
                tot += _ex_uv(K, w[u] * w[v] / W, d, T)
    return tot / n


@pytest.mark.parametrize("d,T", [(1, 0.0), (2, 0.0), (1, 0.5), (2, 0.3), (3, 0.7), (4, 0.9),
                                 (1, 0.05), (2, 0.1), (3, 0.02)])
def test_degree_formula_matches_integration(d, T):
    """Small T included: there c = K^(1/T) leaves the range of doubles and the sums of
    w^(1/T) over all pairs overflow, which the log-domain suffix sums avoid."""
    rng = np.random.default_rng(100 + d)
    w = 1.0 + rng.pareto(1.3, 25)
    W = O.exact_sum(w)
    for K in (1e-3, 0.05, 0.6, 8.0):
        ref = _brute_force_degree(K, w, d, T)
        got = O.girg_avg_degree(None, w, d, T, W, K=K)
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-12), (K, got, ref)


@pytest.mark.parametrize("d,T", [(1, 0.5), (2, 0.0), (2, 0.7), (2, 0.06), (3, 0.15)])
def test_degree_formula_matches_monte_carlo(d, T):
    n, runs = 300, 200
    w, _ = O.girg_points(n, d, 2.5, 1.0, 5)
    W = O.exact_sum(w)
    K = O.girg_solve_K(6.0, w, d, T, W)
    degs = []
    for s in range(runs):
        _, X = O.girg_points(n, d, 2.5, 1.0, 1000 + s)  # fresh positions, same weights
        e = O.girg_allpairs(X, w, W, T, None, 77 + s, K=K)
        degs.append(2.0 * len(e) / n)
    degs = np.array(degs)
    se = degs.std(ddof=1) / math.sqrt(runs)
    assert abs(degs.mean() - 6.0) < 4.5 * se + 1e-9


@pytest.mark.parametrize("d,T,target", [(1, 0.5, 10.0), (2, 0.5, 10.0), (3, 0.7, 16.0),
                                        (2, 0.0, 16.0), (4, 0.0, 16.0), (3, 0.01, 16.0),
                                        (1, 0.9, 4.0)])
def test_solver_inverts_degree(d, T, target):
    w, _ = O.girg_points(20000, d, 2.2, 1.0, 9)
    W = O.exact_sum(w)
    K = O.girg_solve_K(target, w, d, T, W)
    assert K > 0
    assert O.girg_avg_degree(None, w, d, T, W, K=K) == pytest.approx(target, rel=1e-10)


def test_scale_and_c_agree_where_c_is_representable():
    """K = c^T: the same sampler output through c and through K (moderate T)."""
    w, X = O.girg_points(3000, 2, 2.5, 1.0, 4)
    W = O.exact_sum(w)
    c = O.girg_solve_c(8.0, w, 2, 0.5, W)
    K = O.K_of_c(c, 2, 0.5)
    a = O.girg_allpairs(X, w, W, 0.5, c, 3)
    b = O.girg_allpairs(X, w, W, 0.5, None, 3, K=K)
    assert np.array_equal(a, b)
    assert K == pytest.approx(c ** 0.5, rel=1e-15)
