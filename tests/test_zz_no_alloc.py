"""girg_allpairs_noalloc, the entry point for callers that cannot allocate device
memory (a plug-in whose host application owns the device memory pool, a
latency-critical loop where an allocation could block or fail): its edges equal
those of girg_allpairs, on two calls in a row with different inputs, so nothing
stale survives in the shared fixed scratch between calls.  This file is collected
last on purpose."""
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
    Xg = torch.from_numpy(np.ascontiguousarray(X.T).view(np.int32)).cuda()
    return Xg, torch.from_numpy(w).cuda(), W, c


def test_noalloc_matches_allpairs_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gg.load()
    for (n, d, T, seed) in [(20_000, 2, 0.5, 3), (9_000, 1, 0.0, 4)]:
        X, w, W, c = _case(n, d, T, seed)
        ref_edges = torch.empty((n * 16, 2), dtype=torch.int32, device="cuda")
        ref = gg.girg_allpairs(ref_edges, X, w, W=W, T=T, c=c, seed=seed)
        assert ref.status == gg.GIRG_OK
        out = torch.zeros((n * 16, 2), dtype=torch.int32, device="cuda")
        got = gg.girg_allpairs_noalloc(out, X, w, W=W, T=T, c=c, seed=seed)
        assert got.status == gg.GIRG_OK, gg.status_string(got.status)
        assert got.num_edges == ref.num_edges > 0
        assert _edge_set(out, got.num_edges) == _edge_set(ref_edges, ref.num_edges)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    lib = gg.load()
    m = ctypes.c_int64(-1)
    st = lib.girg_allpairs_noalloc((1 << 20) + 1, 1, None, None, 1.0, 0.5, 1.0, 1, 0, 4, None,
                                   0, ctypes.byref(m), None)
    assert st == gg.GIRG_E_PARAM and m.value == -1
