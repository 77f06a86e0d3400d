"""GB300-native GIRG / HRG generator (arXiv 1905.06706) -- Python binding.

Argument marshalling only: every step of the sampler runs in the CUDA library
``libgirg_gb300.so`` (built in-tree by :func:`build`), called through its C ABI
(``include/girg_gb300.h``).  Tensors are PyTorch CUDA tensors; their device
pointers and the current CUDA stream are passed to the library.  There is no
CPU fallback: if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

from .build import LIB, build  # noqa: F401

GIRG_OK = 0
GIRG_E_PARAM = 1
GIRG_E_CAPACITY = 2
GIRG_E_CUDA = 3
GIRG_E_RANGE = 4
GIRG_E_INTERNAL = 5
PRECISION_FP32 = 0
PRECISION_FP64 = 1

STAT_NAMES = ("type1_pairs", "coins", "rechecks", "type2_items", "jump_draws",
              "type2_candidates", "rows", "type1_items", "type2_chunks", "edges",
              "kernel_launches", "type1_vertex_refs", "type1_edges", "type2_streams",
              "edge_checksum", "type2_segments", "enum_passes", "type2_entries",
              "type1_entries")
PHASE_NAMES = ("points_reduce", "tables", "sort", "enumerate", "type1", "type2",
               "total", "host_reduce_readback", "host_c_search", "host_tables")


class GirgParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("beta", ctypes.c_double),
                ("T", ctypes.c_double), ("avg_deg", ctypes.c_double), ("c", ctypes.c_double),
                ("w_min", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("edge_bytes", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("level_cap", ctypes.c_int32)]


class HrgParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("alpha", ctypes.c_double), ("T", ctypes.c_double),
                ("avg_deg", ctypes.c_double), ("R", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("edge_bytes", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("level_cap", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes) of every entry point of include/girg_gb300.h
P, I64, I32, U64, DBL = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                         ctypes.c_double)
SIGNATURES = {
    "girg_generate": (I32, [P, P, I64, P, P, P]),
    "girg_generate_from_points": (I32, [I64, I32, P, P, DBL, DBL, U64, I32, I32, I32, P, I64, P,
                                        P]),
    "hrg_generate": (I32, [P, P, I64, P, P, P]),
    "hrg_expected_avg_degree": (I32, [I64, DBL, DBL, DBL, P]),
    "hrg_solve_radius": (I32, [I64, DBL, DBL, DBL, P]),
    "girg_allpairs": (I32, [I64, I32, P, P, DBL, DBL, DBL, U64, I32, I32, P, I64, P, P]),
    "girg_allpairs_noalloc": (I32, [I64, I32, P, P, DBL, DBL, DBL, U64, I32, I32, P, I64, P,
                                    P]),
    "girg_points": (I32, [I64, I32, DBL, DBL, U64, P, P, P]),
    "hrg_points": (I32, [I64, DBL, DBL, U64, P, P, P]),
    "hrg_girg_points": (I32, [I64, DBL, DBL, U64, P, P, P]),
    "girg_expected_avg_degree": (I32, [P, P, P]),
    "girg_last_stats": (I32, [P, I32]),
    "girg_last_phase_ms": (I32, [P, I32]),
    "girg_sorted_order": (I32, [I64, I32, P, P, DBL, DBL, I32, P, P]),
    "girg_status_string": (ctypes.c_char_p, [I32]),
    "girg_det_eval": (DBL, [I32, DBL, DBL]),
    "girg_last_scale": (DBL, []),
    "girg_expected_edges": (I64, [P, P]),
    "girg_scratch_bytes": (I64, [P]),
    "girg_scratch_pool_usage": (I32, [P, P, P, I32]),
    "girg_scratch_pool_trim": (I32, [I64]),
    "girg_point_cache": (I32, [I64]),
    "girg_point_cache_stats": (I32, [P, P, P, P]),
    "girg_issue_probe": (I32, [I32, I64, P, P, P]),
    "girg_server_create": (I32, [I32, I64, P]),
    "girg_server_submit": (I32, [P, P, P, I64, I64]),
    "girg_server_poll": (I32, [P, P, I32, I32]),
    "girg_server_pending": (I32, [P]),
    "girg_server_clock_us": (DBL, [P]),
    "girg_server_destroy": (I32, [P]),
}


class RequestResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("num_edges", ctypes.c_int64),
                ("c_used", ctypes.c_double), ("checksum", ctypes.c_uint64),
                ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed); raise if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = LIB
        if build_if_missing:
            path = build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgirg_gb300.so not found at {path}; run build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GirgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({status_string(status)})")
        self.status = status


def status_string(status: int) -> str:
    return load().girg_status_string(status).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA GPU is required (this library has no CPU path)")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def last_stats() -> dict:
    buf = (ctypes.c_int64 * len(STAT_NAMES))()
    load().girg_last_stats(buf, len(STAT_NAMES))
    out = dict(zip(STAT_NAMES, list(buf)))
    out["edge_checksum"] &= (1 << 64) - 1  # unsigned
    return out


def girg_expected_edges(*, n, d, beta, T, avg_deg=0.0, c=0.0, w_min=1.0, seed=1,
                        stream=None) -> int:
    """Expected edge count (for sizing the edge buffer)."""
    _torch()
    p = GirgParams(n, d, beta, T, avg_deg, c, w_min, seed, 4, PRECISION_FP32, 0)
    m = load().girg_expected_edges(ctypes.byref(p), _stream(stream))
    if m < 0:
        raise GirgError(GIRG_E_PARAM, "girg_expected_edges")
    return m


def last_K() -> float:
    """The scale K (c^T, or c^d at T = 0) of this thread's last generate call."""
    return load().girg_last_scale()


def scratch_pool_usage(reset_high: bool = False) -> dict:
    """The library's scratch pool on the current device: reserved, used and high-water
    bytes (``reset_high`` resets the high-water mark after reading it)."""
    _torch()
    r, u, h = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().girg_scratch_pool_usage(ctypes.byref(r), ctypes.byref(u), ctypes.byref(h),
                                        1 if reset_high else 0)
    if st != GIRG_OK:
        raise GirgError(st, "girg_scratch_pool_usage")
    return {"reserved": r.value, "used": u.value, "used_high": h.value}


def scratch_pool_trim(keep_bytes: int = 0) -> None:
    """Return the unused memory of the library's scratch pool to the driver."""
    _torch()
    st = load().girg_scratch_pool_trim(keep_bytes)
    if st != GIRG_OK:
        raise GirgError(st, "girg_scratch_pool_trim")


def point_cache(max_bytes: int) -> None:
    """Keep the layouts (sorted points, cell offsets, bound tables) of generated graphs
    on the device, up to max_bytes (0: off), so that repeated requests for the same
    point set skip points, reductions, the scale search and the sort."""
    st = load().girg_point_cache(max_bytes)
    if st != GIRG_OK:
        raise GirgError(st, "girg_point_cache")


def point_cache_stats() -> dict:
    e, b, h, m = (ctypes.c_int64(0) for _ in range(4))
    load().girg_point_cache_stats(ctypes.byref(e), ctypes.byref(b), ctypes.byref(h),
                                  ctypes.byref(m))
    return {"entries": e.value, "bytes": b.value, "hits": h.value, "misses": m.value}


ISSUE_PROBE_KINDS = ("lop3", "imad", "ffma")


def issue_probe(kind: int, iters: int = 2000, stream=None) -> tuple:
    """One launch of the issue-rate probe (kind 0 integer logic, 1 integer multiply-add,
    2 FP32 fused multiply-add): (milliseconds, warp instructions issued by construction)."""
    ms, wi = ctypes.c_float(0.0), ctypes.c_int64(0)
    st = load().girg_issue_probe(kind, iters, _stream(stream), ctypes.byref(ms),
                                 ctypes.byref(wi))
    if st != GIRG_OK:
        raise GirgError(st, "girg_issue_probe")
    return float(ms.value), int(wi.value)


def scratch_bytes(*, n, d, beta, T, avg_deg=0.0, c=0.0, w_min=1.0, seed=1, edge_bytes=4,
                  precision=PRECISION_FP32, level_cap=0) -> int:
    """The server's admission estimate of one request's peak scratch (bytes)."""
    p = GirgParams(n, d, beta, T, avg_deg, c, w_min, seed, edge_bytes, precision, level_cap)
    return load().girg_scratch_bytes(ctypes.byref(p))


def last_phase_ms() -> dict:
    buf = (ctypes.c_float * len(PHASE_NAMES))()
    load().girg_last_phase_ms(buf, len(PHASE_NAMES))
    return dict(zip(PHASE_NAMES, list(buf)))


@dataclass
class Result:
    status: int
    num_edges: int
    c_used: float = float("nan")
    R_used: float = float("nan")


def _edge_args(edges):
    """(edge_bytes, pointer, capacity) of an edge buffer; None means count-only."""
    if edges is None:
        return 0, None, 0
    return edges.element_size(), _ptr(edges), edges.shape[0]


def girg_generate(edges, *, n, d, beta, T, avg_deg=0.0, c=0.0, w_min=1.0, seed=1,
                  precision=PRECISION_FP32, level_cap=0, stream=None) -> Result:
    """Generate a GIRG into ``edges`` ((cap, 2) tensor of int32 or int64: on the GPU, or
    a pinned CPU tensor that the kernels fill directly; None: count-only, see
    ``last_stats()['edge_checksum']``)."""
    _torch()
    lib = load()
    eb, ep, cap = _edge_args(edges)
    p = GirgParams(n, d, beta, T, avg_deg, c, w_min, seed, eb, precision, level_cap)
    m = ctypes.c_int64(0)
    cu = ctypes.c_double(0.0)
    st = lib.girg_generate(ctypes.byref(p), ep, cap, ctypes.byref(m), ctypes.byref(cu),
                           _stream(stream))
    return Result(st, m.value, cu.value)


def girg_generate_from_points(edges, X, w, *, T, c, seed=1, precision=PRECISION_FP32,
                              level_cap=0, stream=None) -> Result:
    """GIRG on caller points: X (d, n) uint32-valued int32/uint32 tensor, w (n,) float64."""
    _torch()
    lib = load()
    d, n = X.shape
    m = ctypes.c_int64(0)
    eb, ep, cap = _edge_args(edges)
    st = lib.girg_generate_from_points(n, d, _ptr(X), _ptr(w), T, c, seed, precision, level_cap,
                                       eb, ep, cap, ctypes.byref(m), _stream(stream))
    return Result(st, m.value, c)


def hrg_generate(edges, *, n, alpha, T, R=0.0, avg_deg=0.0, seed=1, precision=PRECISION_FP32,
                 level_cap=0, stream=None) -> Result:
    """Generate an HRG into ``edges``; R <= 0 solves the radius from ``avg_deg``.
    The radius used is returned in ``R_used``."""
    _torch()
    lib = load()
    eb, ep, cap = _edge_args(edges)
    p = HrgParams(n, alpha, T, avg_deg, R, seed, eb, precision, level_cap)
    m = ctypes.c_int64(0)
    r_used = ctypes.c_double(float("nan"))
    st = lib.hrg_generate(ctypes.byref(p), ep, cap, ctypes.byref(m),
                          ctypes.byref(r_used), _stream(stream))
    return Result(st, m.value, R_used=r_used.value)


def hrg_expected_avg_degree(n, alpha, T, R) -> float:
    """Expected average degree of an HRG (host computation, no GPU needed)."""
    out = ctypes.c_double(0.0)
    st = load().hrg_expected_avg_degree(n, alpha, T, R, ctypes.byref(out))
    if st != GIRG_OK:
        raise GirgError(st, "hrg_expected_avg_degree")
    return out.value


def hrg_solve_radius(n, alpha, T, avg_deg) -> float:
    """Disk radius R with the given expected average degree (host computation)."""
    out = ctypes.c_double(0.0)
    st = load().hrg_solve_radius(n, alpha, T, avg_deg, ctypes.byref(out))
    if st != GIRG_OK:
        raise GirgError(st, "hrg_solve_radius")
    return out.value


def girg_allpairs(edges, X, w, *, W, T, c, seed=1, precision=PRECISION_FP32,
                  stream=None) -> Result:
    _torch()
    lib = load()
    d, n = X.shape
    m = ctypes.c_int64(0)
    st = lib.girg_allpairs(n, d, _ptr(X), _ptr(w), W, T, c, seed, precision,
                           edges.element_size(), _ptr(edges), edges.shape[0], ctypes.byref(m),
                           _stream(stream))
    return Result(st, m.value, c)


def girg_allpairs_noalloc(edges, X, w, *, W, T, c, seed=1, precision=PRECISION_FP32,
                          stream=None) -> Result:
    """girg_allpairs with its scratch in a fixed library-owned device array: for callers
    that cannot allocate device memory (n <= GIRG_NOALLOC_MAX_N = 2^20).  Calls whose
    device work overlaps share that array and must be serialised."""
    _torch()
    lib = load()
    d, n = X.shape
    m = ctypes.c_int64(0)
    st = lib.girg_allpairs_noalloc(n, d, _ptr(X), _ptr(w), W, T, c, seed, precision,
                                   edges.element_size(), _ptr(edges), edges.shape[0],
                                   ctypes.byref(m), _stream(stream))
    return Result(st, m.value, c)


def girg_points(n, d, beta, w_min=1.0, seed=1, stream=None):
    """Weights (n,) float64 and positions (d, n) int32 (uint32 bit patterns)."""
    torch = _torch()
    lib = load()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    X = torch.empty((d, n), dtype=torch.int32, device="cuda")
    st = lib.girg_points(n, d, beta, w_min, seed, _ptr(w), _ptr(X), _stream(stream))
    if st != GIRG_OK:
        raise GirgError(st, "girg_points")
    return w, X


def hrg_points(n, alpha, R, seed=1, stream=None):
    torch = _torch()
    lib = load()
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    X = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.hrg_points(n, alpha, R, seed, _ptr(r), _ptr(X), _stream(stream))
    if st != GIRG_OK:
        raise GirgError(st, "hrg_points")
    return r, X


def hrg_girg_points(n, alpha, R, seed=1, stream=None):
    """The HRG's vertices as GIRG points (Sec. 2.3): weights (n,) float64 and 1-dimensional
    positions (1, n) int32 (uint32 bit patterns)."""
    torch = _torch()
    lib = load()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    X = torch.empty((1, n), dtype=torch.int32, device="cuda")
    st = lib.hrg_girg_points(n, alpha, R, seed, _ptr(w), _ptr(X), _stream(stream))
    if st != GIRG_OK:
        raise GirgError(st, "hrg_girg_points")
    return w, X


def girg_expected_avg_degree(*, n, d, beta, T, c, w_min=1.0, seed=1, stream=None) -> float:
    _torch()
    lib = load()
    p = GirgParams(n, d, beta, T, 0.0, c, w_min, seed, 4, 0, 0)
    out = ctypes.c_double(0.0)
    st = lib.girg_expected_avg_degree(ctypes.byref(p), ctypes.byref(out), _stream(stream))
    if st != GIRG_OK:
        raise GirgError(st, "girg_expected_avg_degree")
    return out.value


def girg_sorted_order(X, w, *, T, c, level_cap=0, stream=None):
    torch = _torch()
    lib = load()
    d, n = X.shape
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    st = lib.girg_sorted_order(n, d, _ptr(X), _ptr(w), T, c, level_cap, _ptr(order),
                               _stream(stream))
    if st != GIRG_OK:
        raise GirgError(st, "girg_sorted_order")
    return order


class Server:
    """Continuous-batching generation server (C++ worker threads, one CUDA stream each).

    ``submit`` queues a request and returns at once; ``poll`` returns finished results
    (``RequestResult``) with server-clock timestamps.  Edge buffers (or None for
    count-only) must stay alive until their result has been polled."""

    def __init__(self, workers=8, memory_budget_bytes=64 << 30):
        _torch()
        self._lib = load()
        self._h = ctypes.c_void_p()
        st = self._lib.girg_server_create(workers, memory_budget_bytes, ctypes.byref(self._h))
        if st != GIRG_OK:
            raise GirgError(st, "girg_server_create")
        self._keep = {}

    def submit(self, request_id, edges, *, n, d, beta, T, avg_deg=0.0, c=0.0, w_min=1.0,
               seed=1, precision=PRECISION_FP32, level_cap=0):
        eb, ep, cap = _edge_args(edges)
        p = GirgParams(n, d, beta, T, avg_deg, c, w_min, seed, eb, precision, level_cap)
        st = self._lib.girg_server_submit(self._h, ctypes.byref(p), ep, cap, request_id)
        if st != GIRG_OK:
            raise GirgError(st, "girg_server_submit")
        self._keep[request_id] = edges

    def poll(self, max_results=1024, wait_for=0):
        buf = (RequestResult * max_results)()
        k = self._lib.girg_server_poll(self._h, buf, max_results, wait_for)
        if k < 0:
            raise GirgError(-k, "girg_server_poll")
        out = [buf[i] for i in range(k)]
        for r in out:
            self._keep.pop(r.request_id, None)
        return out

    def pending(self):
        return self._lib.girg_server_pending(self._h)

    def clock_us(self):
        return self._lib.girg_server_clock_us(self._h)

    def close(self):
        if self._h:
            self._lib.girg_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

