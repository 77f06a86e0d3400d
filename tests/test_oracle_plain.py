"""Pins of the plain build of the oracle (the C library's log, exp, log1p, pow, sin
and acosh in place of the fixed-point functions) and of the decision audit.

* The plain samplers satisfy the same brute-force and statistical pins as the default
  build: every pair covered exactly once, p <= pbar on every type-II pair, the T = 0
  cell-pair sampler equal to all pairs, type-I coins shared with all pairs, the law of
  the geometric jump and per-pair edge frequencies (Sec. 3.2, 3.3, App. B.1).
* The default and plain builds, on the same inputs, give the same graph except for
  decisions the audit marks as near (both sides within a relative 1e-12): the fixed-point
  functions and the C library's round differently, nothing else differs.
* The audit itself: it counts every decision (n (n - 1) / 2 for all pairs) and records a
  decision placed on its threshold.
"""
import math

import numpy as np
import pytest

import oracle as O


def _instance(n, d, beta=2.5, seed=3):
    w, X = O.girg_points(n, d, beta, 1.0, seed, plain=True)
    return w, X, O.exact_sum(w, plain=True)


def _torus_D(X, u, v):
    d = X.shape[1]
    return max(min((int(X[u, k]) - int(X[v, k])) % 2 ** 32,
                   (int(X[v, k]) - int(X[u, k])) % 2 ** 32) for k in range(d))


def _item_pairs(it, order, k):
    a_ids = order[it["a_lo"][k]:it["a_hi"][k]]
    b_ids = order[it["b_lo"][k]:it["b_hi"][k]]
    if it["tri"][k]:
        for x in range(len(a_ids)):
            for y in range(x + 1, len(b_ids)):
                yield a_ids[x], b_ids[y]
    else:
        for u in a_ids:
            for v in b_ids:
                yield u, v


def test_plain_functions_are_the_c_library():
    """The plain build evaluates the paper's formulas with the platform's functions:
    where the fixed-point method rounds differently, the plain build agrees with libm."""
    xs = np.random.default_rng(1).uniform(1e-3, 50.0, 500)
    diff = 0
    for x in xs:
        assert O.det_log(x, plain=True) == math.log(x)
        assert O.det_exp(-x / 10, plain=True) == math.exp(-x / 10)
        assert O.det_pow(x, 0.37, plain=True) == x ** 0.37
        assert O.det_acosh(1.0 + x, plain=True) == math.acosh(1.0 + x)
        diff += O.det_pow(x, 0.37) != x ** 0.37
    assert O.det_log1p(-0.3, plain=True) == math.log1p(-0.3)
    assert O.det_sinpi(0.1, plain=True) == math.sin(math.pi * 0.1)
    # the two builds are different functions (otherwise the check below is empty)
    assert diff > 0


@pytest.mark.parametrize("d,T,lcap", [(1, 0.7, 9), (2, 0.5, 5), (3, 0.6, 4)])
def test_plain_partition_and_bound(d, T, lcap):
    n = 80
    w, X, W = _instance(n, d, beta=2.2, seed=70 + d)
    for c in (0.002, 0.2, 5.0):
        res = O.girg_cellpairs(X, w, 1.0, W, T, c, 1, want_items=True, skip_sampling=True,
                               level_cap=lcap, plain=True)
        cnt = np.zeros((n, n), dtype=np.int64)
        it = res.items
        for k in range(len(it["type"])):
            for u, v in _item_pairs(it, res.order, k):
                cnt[min(u, v), max(u, v)] += 1
                if it["type"][k] == 2:
                    p = O.girg_p(d, T, c, W, w[u], w[v], _torus_D(X, u, v), plain=True)
                    assert p <= it["pbar"][k]
        iu = np.triu_indices(n, 1)
        assert np.all(cnt[iu] == 1)


@pytest.mark.parametrize("d,n", [(1, 6000), (2, 2500)])
def test_plain_threshold_cellpairs_equals_allpairs(d, n):
    w, X, W = _instance(n, d, seed=80 + d)
    c = O.girg_solve_c(10.0, w, d, 0.0, W, plain=True)
    e1 = O.girg_allpairs(X, w, W, 0.0, c, 1, plain=True)
    e2 = O.girg_cellpairs(X, w, 1.0, W, 0.0, c, 1, plain=True).edges
    assert len(e1) > 0
    assert O.edge_set(e1) == O.edge_set(e2)


def test_plain_type1_pairs_share_coins_with_allpairs():
    n, d, T = 1500, 2, 0.7
    w, X, W = _instance(n, d, seed=91)
    c = O.girg_solve_c(8.0, w, d, T, W, plain=True)
    e1 = O.edge_set(O.girg_allpairs(X, w, W, T, c, 7, plain=True))
    res = O.girg_cellpairs(X, w, 1.0, W, T, c, 7, want_items=True, plain=True)
    e2 = O.edge_set(res.edges)
    it = res.items
    t1 = set()
    for k in np.nonzero(it["type"] == 1)[0]:
        for u, v in _item_pairs(it, res.order, k):
            t1.add(min(u, v) * (1 << 32) + max(u, v))
    assert len(t1) > 0 and (e1 & t1) == (e2 & t1)


@pytest.mark.parametrize("pbar", [0.5, 0.01])
def test_plain_geometric_jump_law(pbar):
    N = 300_000
    rng = np.random.default_rng(int(pbar * 1e6) + 11)
    lo = rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
    X = O.geometric_jumps(pbar, lo, hi, plain=True)
    q = 1.0 - pbar
    mean, var = q / pbar, q / pbar ** 2
    assert abs(X.mean() - mean) < 6.0 * math.sqrt(var / N)
    for k in (1, 3, round(2 / pbar)):
        pk = q ** k
        assert abs((X >= k).mean() - pk) < 6.0 * math.sqrt(pk * (1 - pk) / N) + 1e-12


def test_plain_edge_frequencies_match_p():
    n, d, T, c = 12, 2, 0.7, 0.1
    w, X, W = _instance(n, d, beta=2.3, seed=62)
    pmat = np.zeros((n, n))
    for u in range(n):
        for v in range(u + 1, n):
            pmat[u, v] = O.girg_p(d, T, c, W, w[u], w[v], _torus_D(X, u, v), plain=True)
    S = 12000
    counts = np.zeros((n, n))
    for s in range(1, S + 1):
        e = O.girg_cellpairs(X, w, 1.0, W, T, c, s, cap=256, plain=True).edges.astype(np.int64)
        if len(e):
            counts[e[:, 0], e[:, 1]] += 1
    iu = np.triu_indices(n, 1)
    p, f = pmat[iu], counts[iu] / S
    sd = np.sqrt(np.maximum(p * (1 - p), 1e-12) / S)
    assert np.all(np.abs(f - p) <= (4.0 + math.log(len(p)) / 2) * sd + 1.0 / S)


def _compare_builds(run):
    """Run one sampler in the default and the plain build under the audit; return the
    symmetric difference of the edge sets and the plain build's audit."""
    with O.audit(plain=True) as ap:
        e_plain = O.edge_set(run(True))
    with O.audit(plain=False) as ad:
        e_det = O.edge_set(run(False))
    return e_plain ^ e_det, ap, ad


@pytest.mark.parametrize("d,T", [(1, 0.7), (2, 0.5), (3, 0.3), (2, 0.0)])
def test_builds_differ_only_in_near_decisions_girg(d, T):
    n = {1: 30000, 2: 20000, 3: 8000}[d]
    w, X, W = _instance(n, d, seed=100 + d)
    K = O.girg_solve_K(10.0, w, d, T, W, plain=True)
    diff, ap, ad = _compare_builds(
        lambda plain: O.girg_cellpairs(X, w, 1.0, W, T, None, 5, cap=n * 16, K=K,
                                       plain=plain).edges)
    assert ap.decisions == ad.decisions > n
    near = ap.pairs() | ad.pairs()
    assert diff <= near, (len(diff), ap.count)
    assert len(diff) <= 1e-9 * ap.decisions + len(near)


def test_builds_differ_only_in_near_decisions_hrg():
    n, alpha, T = 20000, 0.75, 0.5
    R = 2 * math.log(n) + 1.0
    r, X = O.hrg_points(n, alpha, R, 4, plain=True)
    diff, ap, ad = _compare_builds(
        lambda plain: O.hrg_cellpairs(X, r, R, T, 4, cap=n * 16, plain=plain).edges)
    assert ap.decisions > n
    assert diff <= (ap.pairs() | ad.pairs())


def test_audit_counts_every_decision_and_records_a_tie():
    n, d, T = 300, 2, 0.5
    w, X, W = _instance(n, d, seed=7)
    K = O.girg_solve_K(8.0, w, d, T, W, plain=True)
    with O.audit(plain=True) as a:
        O.girg_allpairs(X, w, W, T, None, 3, K=K, plain=True)
    assert a.decisions == n * (n - 1) // 2
    # place the decision of one pair on its threshold: p_uv = U_uv, from
    # p = (K q / r^d)^(1/T), i.e. K = U^T r^d / q (rounding leaves a few ulps)
    u, v = 10, 200
    D = _torus_D(X, u, v)
    U = O.pair_coin(3, u, v, plain=True)
    q = w[u] * w[v] / W
    K_tie = U ** T * (D * 2.0 ** -32) ** d / q
    p = O.girg_p(d, T, None, W, w[u], w[v], D, K=K_tie, plain=True)
    assert abs(p - U) <= 1e-13 * U
    with O.audit(plain=True) as b:
        O.girg_allpairs(X, w, W, T, None, 3, K=K_tie, plain=True)
    assert (u << 32) + v in b.pairs(kinds=(1,))
    assert b.count < 50  # only decisions this close are recorded
