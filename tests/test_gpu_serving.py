"""The continuous-batching server: every request's graph is the same alone and in
the mix (edge count and order-independent checksum, and the edge set itself for a
few), with requests of mixed size, dimension, exponent, temperature and degree."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1905_06706_gb300 as gg

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
