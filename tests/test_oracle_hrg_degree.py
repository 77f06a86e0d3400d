"""Pins of the oracle's HRG expected degree and its search for R.

The paper gives no formula for the average degree of an HRG (Sec. 2.2 says only
that R = 2 ln n + C with C setting it).  The oracle integrates the model's
definition; these tests tie it to things fixed independently of that code:
Monte Carlo over random vertex pairs, adaptive quadrature of the threshold case,
the large-R limit of the average degree known for the threshold model
(8 alpha^2 nu / (pi (2 alpha - 1)^2), nu = n e^(-R/2)) and the temperature factor
pi T / sin(pi T) of the binomial model.
"""
import math

import numpy as np
import pytest

import oracle as O


def _mc_edge_prob(alpha, T, R, n_pairs, seed):
    rng = np.random.default_rng(seed)
    u = rng.random((2, n_pairs))
    r = np.arccosh(1.0 + u * (math.cosh(alpha * R) - 1.0)) / alpha
    dth = math.pi * rng.random(n_pairs)  # angle difference in [0, pi]
    coshd = np.cosh(r[0] - r[1]) + 2.0 * np.sinh(r[0]) * np.sinh(r[1]) * np.sin(dth / 2) ** 2
    d = np.arccosh(np.maximum(coshd, 1.0))
    if T == 0.0:
        p = (d < R).astype(np.float64)
    else:
        p = 1.0 / (np.exp((d - R) / (2.0 * T)) + 1.0)
    return p.mean(), p.std() / math.sqrt(n_pairs)


@pytest.mark.parametrize("alpha,T,R", [(0.75, 0.0, 10.0), (0.75, 0.3, 10.0), (0.75, 0.7, 12.0),
                                       (1.2, 0.5, 9.0)])
def test_edge_probability_monte_carlo(alpha, T, R):
    n = 1000
    exact = O.hrg_avg_degree(n, alpha, T, R) / (n - 1)
    mean, se = _mc_edge_prob(alpha, T, R, 4_000_000, seed=int(100 * alpha + 10 * T + R))
    assert abs(mean - exact) < 5.0 * se, (mean, exact, se)


def test_threshold_model_against_adaptive_quadrature():
    """T = 0: G(R) by nested adaptive QUADPACK integration of the same definition."""
    integrate = pytest.importorskip("scipy.integrate")
    alpha, R = 0.75, 10.0
    chR = math.cosh(alpha * R) - 1.0

    def f(r):  # radial density
        return alpha * math.sinh(alpha * r) / chR

    def phi(r1, r2):  # fraction of angle differences with dist < R
        if R >= r1 + r2:
            return 1.0
        if R <= abs(r1 - r2):
            return 0.0
        s = (math.cosh(R) - math.cosh(r1 - r2)) / (2.0 * math.sinh(r1) * math.sinh(r2))
        return 2.0 / math.pi * math.asin(math.sqrt(min(max(s, 0.0), 1.0)))

    def inner(r1):
        pts = [x for x in (R - r1,) if 0.0 < x < R]
        v, _ = integrate.quad(lambda r2: f(r2) * phi(r1, r2), 0.0, R, points=pts or None,
                              limit=400, epsabs=0.0, epsrel=1e-12)
        return f(r1) * v

    ref, _ = integrate.quad(inner, 0.0, R, limit=400, epsabs=0.0, epsrel=1e-11)
    got = O.hrg_avg_degree(2, alpha, 0.0, R)
    assert abs(got - ref) <= 1e-9 * ref


@pytest.mark.parametrize("alpha", [0.75, 0.9])
def test_threshold_model_large_R_limit(alpha):
    n = 10 ** 6
    prev = None
    for R, tol in ((40.0, 2e-3), (60.0, 3e-5)):
        nu = n * math.exp(-R / 2.0)
        lim = 8.0 * alpha * alpha * nu / (math.pi * (2.0 * alpha - 1.0) ** 2)
        dev = abs(O.hrg_avg_degree(n, alpha, 0.0, R) / lim - 1.0)
        assert dev < tol
        if prev is not None:
            assert dev < prev  # converges
        prev = dev


@pytest.mark.parametrize("T", [0.3, 0.5])
def test_temperature_factor(T):
    n, alpha, R = 10 ** 6, 0.75, 60.0
    ratio = O.hrg_avg_degree(n, alpha, T, R) / O.hrg_avg_degree(n, alpha, 0.0, R)
    assert abs(ratio / (math.pi * T / math.sin(math.pi * T)) - 1.0) < 1e-4


def test_degree_decreases_in_R_and_search_inverts():
    n, alpha, T = 10 ** 7, 0.75, 0.5
    vals = [O.hrg_avg_degree(n, alpha, T, R) for R in (28.0, 30.0, 32.0, 34.0)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    R = O.hrg_solve_R(n, alpha, T, 10.0)
    assert abs(O.hrg_avg_degree(n, alpha, T, R) - 10.0) < 1e-9 * 10.0
    R0 = O.hrg_solve_R(10 ** 4, 0.75, 0.0, 8.0)
    assert abs(O.hrg_avg_degree(10 ** 4, 0.75, 0.0, R0) - 8.0) < 1e-9 * 8.0
