"""Pins of the cell-pair oracle (Algorithm 1) by brute force and statistics.

* Partition: every unordered vertex pair lies in exactly one item
  (App. B.1), for d = 1..4 (GIRG) and the HRG mapping, with levels forced
  deep; at T = 0 every pair outside the type-I items is a non-edge.
* Bound: p_uv <= pbar for every pair of every type-II item (Sec. 3.2).
* Exactness at T = 0: the cell-pair oracle equals the all-pairs oracle.
* Type-I coins: on type-I pairs the two oracles take the same decisions.
* Distribution: per-pair edge frequencies over 20 000 seeds match p_uv
  (binomial z-test, Bonferroni), which exercises geometric jumps, chunking and
  the p / pbar acceptance.
"""
import math

import numpy as np
import pytest

import oracle as O


def _instance(n, d, beta=2.5, seed=3):
    w, X = O.girg_points(n, d, beta, 1.0, seed)
    return w, X, O.exact_sum(w)


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


def _coverage(res, n):
    it = res.items
    cnt = np.zeros((n, n), dtype=np.int64)
    typ = np.zeros((n, n), dtype=np.int64)
    for k in range(len(it["type"])):
        for u, v in _item_pairs(it, res.order, k):
            a, b = min(u, v), max(u, v)
            assert a != b
            cnt[a, b] += 1
            typ[a, b] = it["type"][k]
    return cnt, typ


@pytest.mark.parametrize("d,T,lcap", [(1, 0.5, 0), (1, 0.7, 9), (2, 0.5, 5), (2, 0.3, 0),
                                      (3, 0.6, 4), (4, 0.5, 3)])
def test_partition_every_pair_exactly_once(d, T, lcap):
    n = 70
    w, X, W = _instance(n, d, seed=10 + d)
    seen = set()
    for c in (0.001, 0.05, 1.0, 30.0):
        res = O.girg_cellpairs(X, w, 1.0, W, T, c, 1, want_items=True, skip_sampling=True,
                               level_cap=lcap)
        cnt, typ = _coverage(res, n)
        iu = np.triu_indices(n, 1)
        assert np.all(cnt[iu] == 1)
        assert np.all(np.tril(cnt) == 0)
        seen |= set(np.unique(typ[iu]).tolist())
    assert seen == {1, 2}


def test_partition_threshold_uncovered_pairs_are_non_edges():
    for d in (1, 2, 3):
        n = 90
        w, X, W = _instance(n, d, seed=20 + d)
        for c in (0.1, 1.0, 3.0):
            res = O.girg_cellpairs(X, w, 1.0, W, 0.0, c, 1, want_items=True, skip_sampling=True)
            cnt, _ = _coverage(res, n)
            assert cnt.max() <= 1
            for u in range(n):
                for v in range(u + 1, n):
                    if cnt[u, v] == 0:
                        D = max(min((int(X[u, k]) - int(X[v, k])) % 2 ** 32,
                                    (int(X[v, k]) - int(X[u, k])) % 2 ** 32) for k in range(d))
                        assert not O.girg_thresh_edge(d, c, W, w[u], w[v], D)


def _torus_D(X, u, v):
    d = X.shape[1]
    return max(min((int(X[u, k]) - int(X[v, k])) % 2 ** 32,
                   (int(X[v, k]) - int(X[u, k])) % 2 ** 32) for k in range(d))


@pytest.mark.parametrize("d,T", [(1, 0.5), (2, 0.7), (3, 0.4), (4, 0.9)])
def test_type2_bound_holds(d, T):
    n = 120
    w, X, W = _instance(n, d, beta=2.2, seed=30 + d)
    checked = 0
    for c in (0.0005, 0.02, 0.2, 5.0):
        res = O.girg_cellpairs(X, w, 1.0, W, T, c, 1, want_items=True, skip_sampling=True,
                               level_cap=8 // d + 1)
        it = res.items
        for k in np.nonzero(it["type"] == 2)[0]:
            pbar = it["pbar"][k]
            assert 0.0 < pbar <= 1.0
            for u, v in _item_pairs(it, res.order, k):
                p = O.girg_p(d, T, c, W, w[u], w[v], _torus_D(X, u, v))
                assert p <= pbar
                checked += 1
    assert checked > 100


@pytest.mark.parametrize("d,n", [(1, 10000), (2, 3000), (3, 3000)])
def test_threshold_cellpairs_equals_allpairs(d, n):
    w, X, W = _instance(n, d, seed=40 + d)
    c = O.girg_solve_c(10.0, w, d, 0.0, W)
    e1 = O.girg_allpairs(X, w, W, 0.0, c, 1)
    e2 = O.girg_cellpairs(X, w, 1.0, W, 0.0, c, 1).edges
    assert len(e1) > 0
    assert O.edge_set(e1) == O.edge_set(e2)


@pytest.mark.parametrize("d,T", [(1, 0.5), (2, 0.7)])
def test_type1_pairs_share_coins_with_allpairs(d, T):
    n = 1500
    w, X, W = _instance(n, d, seed=50 + d)
    c = O.girg_solve_c(8.0, w, d, T, W)
    e1 = O.edge_set(O.girg_allpairs(X, w, W, T, c, 7))
    res = O.girg_cellpairs(X, w, 1.0, W, T, c, 7, want_items=True)
    e2 = O.edge_set(res.edges)
    it = res.items
    t1 = set()
    for k in np.nonzero(it["type"] == 1)[0]:
        for u, v in _item_pairs(it, res.order, k):
            t1.add(min(u, v) * (1 << 32) + max(u, v))
    assert len(t1) > 0
    assert (e1 & t1) == (e2 & t1)
    # and the oracle's edges outside type-I pairs come from type-II items
    assert len(e2 - t1) == res.stats["type2_edges"]


def _frequency_test(run, pmat, n_seeds, n):
    counts = np.zeros((n, n))
    for s in range(1, n_seeds + 1):
        e = run(s)
        if len(e):
            counts[e[:, 0], e[:, 1]] += 1
    iu = np.triu_indices(n, 1)
    p = pmat[iu]
    f = counts[iu] / n_seeds
    m = len(p)
    z = 4.0 + math.log(m) / 2  # Bonferroni-style margin
    sd = np.sqrt(np.maximum(p * (1 - p), 1e-12) / n_seeds)
    assert np.all(np.abs(f - p) <= z * sd + 1.0 / n_seeds), np.max(np.abs(f - p) / sd)
    return f, p


@pytest.mark.parametrize("d,T,c", [(1, 0.5, 0.3), (2, 0.7, 0.1), (2, 0.4, 0.03)])
def test_girg_edge_frequencies_match_p(d, T, c):
    n = 14
    w, X, W = _instance(n, d, beta=2.3, seed=60 + d)
    pmat = np.zeros((n, n))
    for u in range(n):
        for v in range(u + 1, n):
            pmat[u, v] = O.girg_p(d, T, c, W, w[u], w[v], _torus_D(X, u, v))
    # levels down to (bitlen(n) + 4) / d, so that most pairs go through geometric jumps
    lcap = 8 // d
    res = O.girg_cellpairs(X, w, 1.0, W, T, c, 1, want_items=True, skip_sampling=True,
                           level_cap=lcap)
    cnt, typ = _coverage(res, n)
    assert (typ == 2).sum() >= 25  # most pairs go through geometric jumps

    def run(s):
        return O.girg_cellpairs(X, w, 1.0, W, T, c, s, cap=256,
                                level_cap=lcap).edges.astype(np.int64)

    _frequency_test(run, pmat, 20000, n)


def test_hrg_edge_frequencies_match_p():
    n, alpha, T = 14, 0.75, 0.5
    R = 2 * math.log(n) + 1.0
    r, X = O.hrg_points(n, alpha, R, 9)
    pmat = np.zeros((n, n))
    for u in range(n):
        for v in range(u + 1, n):
            D = min((int(X[u]) - int(X[v])) % 2 ** 32, (int(X[v]) - int(X[u])) % 2 ** 32)
            pmat[u, v] = O.hrg_p(T, R, r[u], r[v], D)

    def run(s):
        return O.hrg_cellpairs(X, r, R, T, s, cap=256).edges.astype(np.int64)

    _frequency_test(run, pmat, 20000, n)


def test_hrg_partition_bound_and_threshold_equality():
    n, alpha = 80, 0.75
    R = 2 * math.log(n) + 0.5
    r, X = O.hrg_points(n, alpha, R, 17)
    for T in (0.3, 0.8):
        res = O.hrg_cellpairs(X, r, R, T, 1, want_items=True, skip_sampling=True, level_cap=6)
        cnt, typ = _coverage(res, n)
        iu = np.triu_indices(n, 1)
        assert np.all(cnt[iu] == 1)
        assert (typ[iu] == 2).sum() > 0
        it = res.items
        for k in np.nonzero(it["type"] == 2)[0]:
            for u, v in _item_pairs(it, res.order, k):
                D = min((int(X[u]) - int(X[v])) % 2 ** 32, (int(X[v]) - int(X[u])) % 2 ** 32)
                assert O.hrg_p(T, R, r[u], r[v], D) <= it["pbar"][k]
    n = 4000
    R = 2 * math.log(n) + 1.0
    r, X = O.hrg_points(n, alpha, R, 18)
    e1 = O.hrg_allpairs(X, r, R, 0.0, 1)
    e2 = O.hrg_cellpairs(X, r, R, 0.0, 1).edges
    assert len(e1) > 1000
    assert O.edge_set(e1) == O.edge_set(e2)


@pytest.mark.parametrize("pbar", [0.9, 0.5, 0.1, 0.01, 1e-4])
def test_geometric_jump_law(pbar):
    """Sec. 3.2: the jump between candidates is geometric: P(X >= k) = (1 - pbar)^k,
    mean (1 - pbar) / pbar, variance (1 - pbar) / pbar^2.  A wrong log, sign, rounding
    direction or pbar in place of 1 - pbar fails one of these."""
    N = 400_000
    rng = np.random.default_rng(int(pbar * 1e6) + 5)
    lo = rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
    hi = rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
    X = O.geometric_jumps(pbar, lo, hi)
    assert (X >= 0).all()
    q = 1.0 - pbar
    mean, var = q / pbar, q / pbar ** 2
    assert abs(X.mean() - mean) < 6.0 * math.sqrt(var / N)
    assert abs(X.var() / var - 1.0) < 0.045
    for k in sorted({1, 2, 5, round(1 / pbar), round(3 / pbar)}):
        pk = q ** k
        emp = (X >= k).mean()
        assert abs(emp - pk) < 6.0 * math.sqrt(pk * (1.0 - pk) / N) + 1e-12, k
