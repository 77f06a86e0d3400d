"""girg_allpairs_noalloc, the entry point for callers that cannot allocate device
memory (a plug-in whose host application owns the device memory pool, a
latency-critical loop where an allocation could block or fail): its edges equal
those of girg_allpairs and those of the oracle's quadratic generator, on two calls in
a row with different inputs, so nothing stale survives in the shared fixed scratch
between calls; a call takes no device memory; a pointer the GPU cannot use is refused
before any device work.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_06706_gb300 as gg  # noqa: E402


def _edge_set(edges, m):
    e = edges[:m].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    return set((e[:, 0] * (1 << 32) + e[:, 1]).tolist())


def _case(n, d, T, seed):
    w, X = O.girg_points(n, d, 2.5, 1.0, seed)
    W = O.exact_sum(w)
    c = O.girg_solve_c(10.0, w, d, T, W)
    ref = O.edge_set(O.girg_allpairs(X, w, W, T, c, seed))
    Xg = torch.from_numpy(np.ascontiguousarray(X.T).view(np.int32)).cuda()
    return Xg, torch.from_numpy(w).cuda(), W, c, ref


def test_noalloc_matches_allpairs_and_oracle_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gg.load()
    for (n, d, T, seed) in [(20_000, 2, 0.5, 3), (9_000, 1, 0.0, 4)]:
        X, w, W, c, oracle_edges = _case(n, d, T, seed)
        ref_edges = torch.empty((n * 16, 2), dtype=torch.int32, device="cuda")
        ref = gg.girg_allpairs(ref_edges, X, w, W=W, T=T, c=c, seed=seed)
        assert ref.status == gg.GIRG_OK
        out = torch.zeros((n * 16, 2), dtype=torch.int32, device="cuda")
        got = gg.girg_allpairs_noalloc(out, X, w, W=W, T=T, c=c, seed=seed)
        assert got.status == gg.GIRG_OK, gg.status_string(got.status)
        assert got.num_edges == ref.num_edges > 0
        assert _edge_set(out, got.num_edges) == _edge_set(ref_edges, ref.num_edges)
        assert _edge_set(out, got.num_edges) == oracle_edges


def test_noalloc_takes_no_device_memory():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gg.load()
    X, w, W, c, _ = _case(5_000, 2, 0.5, 6)
    out = torch.zeros((5_000 * 16, 2), dtype=torch.int32, device="cuda")
    first = gg.girg_allpairs_noalloc(out, X, w, W=W, T=0.5, c=c, seed=6)  # warm-up
    assert first.status == gg.GIRG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        r = gg.girg_allpairs_noalloc(out, X, w, W=W, T=0.5, c=c, seed=6)
        assert r.status == gg.GIRG_OK and r.num_edges == first.num_edges
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_refuses_pageable_host_memory():
    lib = gg.load()
    X, w, W, c, _ = _case(2_000, 1, 0.5, 8)
    host = np.zeros((2_000 * 16, 2), dtype=np.int32)  # pageable: the GPU cannot write it
    m = ctypes.c_int64(-1)
    st = lib.girg_allpairs_noalloc(2_000, 1, X.data_ptr(), w.data_ptr(), W, 0.5, c, 8, 0, 4,
                                   host.ctypes.data, len(host), ctypes.byref(m), None)
    assert st == gg.GIRG_E_PARAM and m.value == -1
    assert not host.any()


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    lib = gg.load()
    m = ctypes.c_int64(-1)
    st = lib.girg_allpairs_noalloc((1 << 20) + 1, 1, None, None, 1.0, 0.5, 1.0, 1, 0, 4, None,
                                   0, ctypes.byref(m), None)
    assert st == gg.GIRG_E_PARAM and m.value == -1
