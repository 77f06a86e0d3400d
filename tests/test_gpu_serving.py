"""The continuous-batching server: every request's graph is the same alone and in
the mix (edge count and order-independent checksum, and the edge set itself for a
few), with requests of mixed size, dimension, exponent, temperature and degree; in the
mix, requests equal the oracle's cell-pair sampler edge for edge; the admission
estimate of a request's scratch is at least the scratch it actually takes."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
import paper_1905_06706_gb300 as gg  # noqa: E402

pytestmark = pytest.mark.gpu


def _mixed_requests(k, seed, n_max=200_000):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(k):
        reqs.append(dict(n=int(math.exp(rng.uniform(math.log(1e3), math.log(n_max)))),
                         d=int(rng.integers(1, 4)), beta=float(rng.uniform(2.1, 3.0)),
                         T=float(rng.uniform(0.0, 0.9)) if r % 5 else 0.0,
                         avg_deg=float(math.exp(rng.uniform(math.log(4), math.log(32)))),
                         seed=1000 + r))
    return reqs


def _cap(q):
    return int(q["n"] * q["avg_deg"] * 1.5) + 4096


def _alone(q, with_edges=True):
    ed = torch.empty((_cap(q), 2), dtype=torch.int32, device="cuda") if with_edges else None
    r = gg.girg_generate(ed, **q)
    assert r.status == gg.GIRG_OK
    cs = gg.last_stats()["edge_checksum"]
    torch.cuda.synchronize()
    return r.num_edges, cs, ed


def test_results_equal_alone_and_in_the_mix():
    reqs = _mixed_requests(40, 5)
    alone = [_alone(q, with_edges=False)[:2] for q in reqs]
    bufs = [torch.empty((_cap(q), 2), dtype=torch.int32, device="cuda") for q in reqs]
    torch.cuda.synchronize()
    with gg.Server(workers=8, memory_budget_bytes=8 << 30) as srv:
        for i, q in enumerate(reqs):
            srv.submit(i, bufs[i] if i % 3 else None, **q)  # every third request count-only
        got = {}
        while len(got) < len(reqs):
            for r in srv.poll(64, wait_for=1):
                got[r.request_id] = r
    for i, q in enumerate(reqs):
        r = got[i]
        assert r.status == gg.GIRG_OK, (i, q, r.status)
        assert (r.num_edges, r.checksum) == alone[i], (i, q)
        assert r.t_submit_us <= r.t_start_us <= r.t_done_us
    # the stored edges themselves, for a few requests
    for i in (1, 2, 4, 5):
        m, cs, ed = _alone(reqs[i])
        a = ed[:m].cpu().numpy()
        b = bufs[i][:got[i].num_edges].cpu().numpy()
        ka = np.sort(a[:, 0].astype(np.int64) << 32 | a[:, 1])
        kb = np.sort(b[:, 0].astype(np.int64) << 32 | b[:, 1])
        assert np.array_equal(ka, kb)


def test_tiny_budget_runs_one_at_a_time():
    reqs = _mixed_requests(6, 9, n_max=30_000)
    alone = [_alone(q, with_edges=False)[:2] for q in reqs]
    with gg.Server(workers=4, memory_budget_bytes=1) as srv:
        for i, q in enumerate(reqs):
            srv.submit(i, None, **q)
        res = []
        while len(res) < len(reqs):
            res += srv.poll(16, wait_for=1)
    res.sort(key=lambda r: r.t_start_us)
    for a, b in zip(res, res[1:]):
        assert b.t_start_us >= a.t_done_us  # never two at once under a 1-byte budget
    for r in res:
        assert (r.num_edges, r.checksum) == alone[r.request_id]


def test_requests_in_the_mix_equal_the_oracle():
    """Requests with the oracle's c (so both sides use the same scale K) run in a mix
    with others; each stored edge set equals the oracle's cell-pair sampler."""
    reqs = _mixed_requests(24, 11, n_max=60_000)
    checked = [i for i, q in enumerate(reqs) if q["n"] <= 40_000][:5]
    assert len(checked) >= 4
    for i in checked:
        q = reqs[i]
        w, X = O.girg_points(q["n"], q["d"], q["beta"], 1.0, q["seed"])
        W = O.exact_sum(w)
        q["c"] = O.girg_solve_c(q["avg_deg"], w, q["d"], q["T"], W)
        q["_ref"] = O.edge_set(O.girg_cellpairs(X, w, 1.0, W, q["T"], q["c"], q["seed"],
                                                cap=_cap(q)).edges)
    bufs = [torch.empty((_cap(q), 2), dtype=torch.int32, device="cuda") for q in reqs]
    torch.cuda.synchronize()
    with gg.Server(workers=8, memory_budget_bytes=8 << 30) as srv:
        for i, q in enumerate(reqs):
            srv.submit(i, bufs[i], **{k: v for k, v in q.items() if not k.startswith("_")})
        got = {}
        while len(got) < len(reqs):
            for r in srv.poll(64, wait_for=1):
                got[r.request_id] = r
    for i in checked:
        r = got[i]
        assert r.status == gg.GIRG_OK
        e = bufs[i][: r.num_edges].cpu().numpy().astype(np.int64)
        assert set((e[:, 0] * (1 << 32) + e[:, 1]).tolist()) == reqs[i]["_ref"], i


def test_admission_estimate_bounds_the_scratch_taken():
    """The server admits requests by girg_scratch_bytes; each request's actual peak
    scratch (the high-water mark of the library's pool, the request running alone) must
    not exceed it, and a mix under a budget of the largest estimate keeps the pool's
    high-water mark within the budget plus one request."""
    reqs = _mixed_requests(16, 13, n_max=1_000_000)
    est = []
    for q in reqs:
        e = gg.scratch_bytes(**q)
        torch.cuda.synchronize()
        gg.scratch_pool_trim(0)
        gg.scratch_pool_usage(reset_high=True)
        r = gg.girg_generate(None, **q)
        assert r.status == gg.GIRG_OK
        torch.cuda.synchronize()
        peak = gg.scratch_pool_usage()["used_high"]
        print(f"n={q['n']} d={q['d']} T={q['T']:.2f}: peak {peak} estimate {e} "
              f"({peak / e:.2f})")
        assert peak <= e, (q, peak, e)
        est.append(e)
    budget = max(est)
    gg.scratch_pool_usage(reset_high=True)
    with gg.Server(workers=8, memory_budget_bytes=budget) as srv:
        for i, q in enumerate(reqs):
            srv.submit(i, None, **q)
        res = []
        while len(res) < len(reqs):
            res += srv.poll(64, wait_for=1)
    assert all(r.status == gg.GIRG_OK for r in res)
    assert gg.scratch_pool_usage()["used_high"] <= budget


def test_resident_point_sets_give_the_same_graph():
    """With the point cache on, a repeated request samples from the kept layout (no
    points, reductions, scale search or sort on the device) and makes the same graph;
    requests that differ in any input of the layout miss; a small limit evicts."""
    q = dict(n=150_000, d=2, beta=2.5, T=0.5, avg_deg=10.0, seed=77)
    ed0 = torch.empty((_cap(q), 2), dtype=torch.int32, device="cuda")
    r0 = gg.girg_generate(ed0, **q)
    cs0 = gg.last_stats()["edge_checksum"]
    gg.point_cache(4 << 30)
    try:
        for rep in range(3):
            ed = torch.empty((_cap(q), 2), dtype=torch.int32, device="cuda")
            r = gg.girg_generate(ed, **q)
            assert r.status == gg.GIRG_OK and r.num_edges == r0.num_edges
            assert gg.last_stats()["edge_checksum"] == cs0
            ph = gg.last_phase_ms()
            if rep > 0:  # a hit: the points and the sort did not run
                assert ph["points_reduce"] < 0.01 and ph["sort"] < 0.01
        st = gg.point_cache_stats()
        assert st["entries"] == 1 and st["hits"] == 2 and st["misses"] == 1
        a = ed0[: r0.num_edges].cpu().numpy()
        b = ed[: r.num_edges].cpu().numpy()
        assert np.array_equal(np.sort(a[:, 0].astype(np.int64) << 32 | a[:, 1]),
                              np.sort(b[:, 0].astype(np.int64) << 32 | b[:, 1]))
        # a different seed or temperature misses and is a different entry
        gg.girg_generate(None, **dict(q, seed=78))
        gg.girg_generate(None, **dict(q, T=0.6))
        assert gg.point_cache_stats()["entries"] == 3
        # a limit below one layout keeps nothing more and evicts down to the limit
        gg.point_cache(st["bytes"] // 2)
        assert gg.point_cache_stats()["bytes"] <= st["bytes"] // 2
        r = gg.girg_generate(None, **q)
        assert r.num_edges == r0.num_edges and gg.last_stats()["edge_checksum"] == cs0
        # and the server's requests use the cache (once the layout is kept: concurrent
        # first requests all build it)
        gg.point_cache(4 << 30)
        gg.girg_generate(None, **q)
        hits = gg.point_cache_stats()["hits"]
        with gg.Server(workers=4, memory_budget_bytes=8 << 30) as srv:
            for i in range(6):
                srv.submit(i, None, **q)
            res = []
            while len(res) < 6:
                res += srv.poll(16, wait_for=1)
        assert all(x.status == gg.GIRG_OK and x.num_edges == r0.num_edges and
                   x.checksum == cs0 for x in res)
        assert gg.point_cache_stats()["hits"] == hits + 6
    finally:
        gg.point_cache(0)
    assert gg.point_cache_stats()["entries"] == 0
