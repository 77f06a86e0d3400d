"""Parity at the full sizes of the dimension sweep (n = 2^24, beta = 2.2, average degree
16, int64 edges, T in {0, 0.7}, d = 1..4) and of the large HRG (n = 10^7, alpha = 0.75,
T = 0.5, R solved for degree 10), where the oracle's samplers are too slow to produce
the whole graph:

* the same configurations at n = 2^14 .. 2^18 edge for edge against the oracle;
* at full size, FP32 and FP64 decisions give the same graph (count and checksum);
  the edges are valid (u < v < n, no duplicates); the average degree is close to the
  target; at T = 0 the neighbourhoods of sampled vertices equal the oracle's brute
  force over all n vertices.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1905_06706_gb300 as gg  # noqa: E402

pytestmark = pytest.mark.gpu

SWEEP = [(d, T) for T in (0.0, 0.7) for d in (1, 2, 3, 4)]
BETA, DEG = 2.2, 16.0


REDUCED_N = {1: 1 << 18, 2: 1 << 18, 3: 1 << 16, 4: 1 << 14}  # the oracle's time grows with d


@pytest.mark.parametrize("d,T", SWEEP)
def test_sweep_reduced_size_edge_for_edge(d, T):
    n = REDUCED_N[d]
    w, X = O.girg_points(n, d, BETA, 1.0, 3)
    W = O.exact_sum(w)
    K = O.girg_solve_K(DEG, w, d, T, W)
    ed = torch.empty((n * 24, 2), dtype=torch.int64, device="cuda")
    r = gg.girg_generate(ed, n=n, d=d, beta=BETA, T=T, avg_deg=DEG, seed=3)
    assert r.status == gg.GIRG_OK
    assert gg.last_K() == pytest.approx(K, rel=1e-9)
    ref = O.girg_cellpairs(X, w, 1.0, W, T, None, 3, cap=n * 24, K=gg.last_K())
    assert r.num_edges == len(ref.edges)
    assert gg.last_stats()["edge_checksum"] == O.edge_checksum(ref.edges)


def _valid_edges(ed, m, n):
    e = ed[:m]
    assert bool((e[:, 0] < e[:, 1]).all()) and bool((e[:, 0] >= 0).all())
    assert bool((e[:, 1] < n).all())
    key = e[:, 0] * n + e[:, 1]
    assert torch.unique(key).numel() == m  # no multi-edges


@pytest.mark.parametrize("d,T", SWEEP)
def test_sweep_full_size(d, T):
    n = 1 << 24
    ed = torch.empty((int(n * DEG * 0.75), 2), dtype=torch.int64, device="cuda")
    r = gg.girg_generate(ed, n=n, d=d, beta=BETA, T=T, avg_deg=DEG, seed=1)
    assert r.status == gg.GIRG_OK
    K, cs = gg.last_K(), gg.last_stats()["edge_checksum"]
    _valid_edges(ed, r.num_edges, n)
    assert abs(2.0 * r.num_edges / n - DEG) < 0.05 * DEG
    r64 = gg.girg_generate(None, n=n, d=d, beta=BETA, T=T, avg_deg=DEG, seed=1,
                           precision=gg.PRECISION_FP64)
    assert (r64.num_edges, gg.last_stats()["edge_checksum"]) == (r.num_edges, cs)
    if T == 0.0:
        # exact neighbourhoods of sampled vertices by the oracle's brute force
        w, X = O.girg_points(n, d, BETA, 1.0, 1)
        W = O.exact_sum(w)
        us = np.random.default_rng(d).choice(n, size=48, replace=False)
        ref = O.girg_thresh_neighbors(X, w, W, K, us)
        e = ed[: r.num_edges]
        ut = torch.as_tensor(us, device="cuda")
        a = torch.isin(e[:, 0], ut)
        b = torch.isin(e[:, 1], ut)
        got = torch.cat([e[a], e[b][:, [1, 0]]]).cpu().numpy()
        assert set(map(tuple, got.tolist())) == set(map(tuple, ref.tolist()))


def test_large_hrg_full_size():
    n, alpha, T = 10_000_000, 0.75, 0.5
    ed = torch.empty((n * 8, 2), dtype=torch.int32, device="cuda")
    r = gg.hrg_generate(ed, n=n, alpha=alpha, T=T, avg_deg=10.0, seed=1)
    assert r.status == gg.GIRG_OK
    assert r.R_used == pytest.approx(O.hrg_solve_R(n, alpha, T, 10.0), rel=1e-9)
    cs = gg.last_stats()["edge_checksum"]
    _valid_edges(ed.to(torch.int64), r.num_edges, n)
    assert abs(2.0 * r.num_edges / n - 10.0) < 0.1 * 10.0
    r64 = gg.hrg_generate(None, n=n, alpha=alpha, T=T, R=r.R_used, seed=1,
                          precision=gg.PRECISION_FP64)
    assert (r64.num_edges, gg.last_stats()["edge_checksum"]) == (r.num_edges, cs)


def test_large_hrg_reduced_size_edge_for_edge():
    n, alpha, T = 200_000, 0.75, 0.5
    R = O.hrg_solve_R(n, alpha, T, 10.0)
    ed = torch.empty((n * 16, 2), dtype=torch.int32, device="cuda")
    r = gg.hrg_generate(ed, n=n, alpha=alpha, T=T, avg_deg=10.0, seed=2)
    assert r.status == gg.GIRG_OK and r.R_used == pytest.approx(R, rel=1e-9)
    rr, X = O.hrg_points(n, alpha, r.R_used, 2)
    ref = O.hrg_cellpairs(X, rr, r.R_used, T, 2, cap=n * 16)
    assert r.num_edges == len(ref.edges)
    assert gg.last_stats()["edge_checksum"] == O.edge_checksum(ref.edges)


@pytest.mark.parametrize("d,T", [(1, 0.0), (2, 0.7), (3, 0.5)])
def test_scale_search_with_many_top_weights(d, T):
    """At n = 2^21, beta = 2.2 the degree model's top set (weights that can meet an E_R
    partner) holds tens of thousands of weights, more than the one-block sort takes:
    the device radix sort orders them, and the scale K equals the oracle's search."""
    n = 1 << 21
    w, X = O.girg_points(n, d, BETA, 1.0, 5)
    W = O.exact_sum(w)
    K = O.girg_solve_K(DEG, w, d, T, W)
    r = gg.girg_generate(None, n=n, d=d, beta=BETA, T=T, avg_deg=DEG, seed=5)
    assert r.status == gg.GIRG_OK
    assert gg.last_K() == pytest.approx(K, rel=1e-9)
