"""CPU oracle for the GIRG / HRG sampler (arXiv 1905.06706).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It wraps the
plain FP64 C restatement of the paper in ``girg_oracle.c`` (see the header of
that file for what each function follows) with ``ctypes`` and ``numpy``; it
shares no code with the CUDA library.

The C file is compiled on first use (or by :func:`build`) with
``-ffp-contract=off`` so that the deterministic elementary functions give the
same bits on every IEEE machine.  It is compiled twice: the default build uses
the file's fixed-point ln / exp (the method the CUDA library implements too, so
the two take identical decisions), the plain build (``plain=True`` on every
function below) the C library's log, exp, log1p, pow, sin and acosh.  The plain
build shares no elementary function with the CUDA library; :class:`audit`
records the decisions that a different rounding could flip.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "girg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgirg_oracle.so")
_PLAIN_PATH = os.path.join(_BUILD, "libgirg_oracle_plain.so")
_lock = threading.Lock()
_libs = {}

MAXL = 64

# stats indices of the cell-pair oracle
STAT_NAMES = (
    "type1_pairs",
    "type2_items",
    "jump_draws",
    "type2_candidates",
    "type1_items",
    "cell_pairs_visited",
    "type1_edges",
    "type2_edges",
)


def _build_one(path: str, defines, force: bool) -> str:
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *defines, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle's two shared libraries (gcc, FP contraction off): the default
    build and the plain build (-DORC_PLAIN).  Returns the default one's path."""
    os.makedirs(_BUILD, exist_ok=True)
    _build_one(_PLAIN_PATH, ["-DORC_PLAIN"], force)
    return _build_one(_LIB_PATH, [], force)


def _load(plain: bool = False):
    with _lock:
        if plain in _libs:
            return _libs[plain]
        build()
        lib = ctypes.CDLL(_PLAIN_PATH if plain else _LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, u32, u64, dbl = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        sig = {
            "orc_philox": (None, [P, P, P]),
            "orc_uniform": (dbl, [u32, u32]),
            "orc_det_log": (dbl, [dbl]),
            "orc_det_log1p": (dbl, [dbl]),
            "orc_det_exp": (dbl, [dbl]),
            "orc_det_pow": (dbl, [dbl, dbl]),
            "orc_det_sinpi": (dbl, [dbl]),
            "orc_det_acosh": (dbl, [dbl]),
            "orc_exact_sum": (dbl, [i64, P]),
            "orc_girg_points": (None, [i64, i32, dbl, dbl, u64, P, P]),
            "orc_hrg_points": (None, [i64, dbl, dbl, u64, P, P]),
            "orc_hrg_weight": (dbl, [dbl, dbl]),
            "orc_girg_p": (dbl, [i32, dbl, dbl, dbl, dbl, dbl, u32]),
            "orc_girg_thresh_edge": (i32, [i32, dbl, dbl, dbl, dbl, u32]),
            "orc_hrg_coshd": (dbl, [dbl, dbl, u32]),
            "orc_hrg_p": (dbl, [dbl, dbl, dbl, dbl, u32]),
            "orc_pair_coin": (dbl, [u64, u32, u32]),
            "orc_girg_allpairs": (i64, [i64, i32, P, P, dbl, dbl, dbl, u64, P, i64]),
            "orc_hrg_allpairs": (i64, [i64, P, P, dbl, dbl, u64, P, i64]),
            "orc_morton": (u64, [P, i32, i32]),
            "orc_cell_linf": (u32, [u64, u64, i32, i32]),
            "orc_level_cap": (i32, [i64, i32, dbl]),
            "orc_chunk_log": (i32, [dbl]),
            "orc_layer_of": (i32, [dbl, dbl]),
            "orc_geometric_jumps": (None, [i64, dbl, P, P, P]),
            "orc_girg_cellpairs": (i64, [i64, i32, P, P, dbl, dbl, dbl, dbl, u64, P, i64,
                                         P, P, P, P, P, i64, P, i32, i32]),
            "orc_hrg_cellpairs": (i64, [i64, P, P, dbl, dbl, u64, P, i64, P, P, P, P, P,
                                        i64, P, i32, i32]),
            "orc_girg_avg_degree": (dbl, [dbl, i64, i32, dbl, P, dbl]),
            "orc_girg_solve_K": (dbl, [dbl, i64, i32, dbl, P, dbl]),
            "orc_girg_K_of_c": (dbl, [dbl, i32, dbl]),
            "orc_girg_thresh_neighbors": (i64, [i64, i32, P, P, dbl, dbl, P, i64, P, i64]),
            "orc_hrg_avg_degree": (dbl, [i64, dbl, dbl, dbl]),
            "orc_hrg_solve_R": (dbl, [i64, dbl, dbl, dbl]),
            "orc_audit_begin": (None, [dbl, P, i64]),
            "orc_audit_end": (i64, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[plain] = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- primitives

def philox(ctr, key, plain=False):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (4 + 2 words)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load(plain).orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(lo: int, hi: int, plain=False) -> float:
    return _load(plain).orc_uniform(lo, hi)


def det_log(x, plain=False):
    return _load(plain).orc_det_log(float(x))


def det_log1p(x, plain=False):
    return _load(plain).orc_det_log1p(float(x))


def det_exp(x, plain=False):
    return _load(plain).orc_det_exp(float(x))


def det_pow(x, y, plain=False):
    return _load(plain).orc_det_pow(float(x), float(y))


def det_sinpi(x, plain=False):
    return _load(plain).orc_det_sinpi(float(x))


def det_acosh(x, plain=False):
    return _load(plain).orc_det_acosh(float(x))


def exact_sum(w, plain=False) -> float:
    w = np.ascontiguousarray(w, dtype=np.float64)
    return _load(plain).orc_exact_sum(len(w), _ptr(w))


def morton(x, d: int, level: int, plain=False) -> int:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint32))
    return _load(plain).orc_morton(_ptr(x), d, level)


def cell_linf(A: int, B: int, d: int, level: int, plain=False) -> int:
    return _load(plain).orc_cell_linf(A, B, d, level)


def level_cap(n: int, d: int, T: float, plain=False) -> int:
    """The default deepest quadtree level for n vertices in dimension d at temperature T."""
    return _load(plain).orc_level_cap(n, d, T)


def geometric_jumps(pbar: float, lo, hi, plain=False):
    """Jumps X = floor(ln U / ln(1 - pbar)) (Sec. 3.2) from word pairs (lo, hi); -1 marks
    a jump of 2^63 or more."""
    lo = np.ascontiguousarray(lo, dtype=np.uint32)
    hi = np.ascontiguousarray(hi, dtype=np.uint32)
    out = np.zeros(len(lo), dtype=np.int64)
    _load(plain).orc_geometric_jumps(len(lo), float(pbar), _ptr(lo), _ptr(hi), _ptr(out))
    return out


def layer_of(w: float, w_min: float, plain=False) -> int:
    """Weight bucket: floor(log2(w / w_min)) of the FP64 quotient, clamped to [0, 63]."""
    return _load(plain).orc_layer_of(float(w), float(w_min))


def chunk_log(pbar: float, plain=False) -> int:
    return _load(plain).orc_chunk_log(pbar)


def pair_coin(seed: int, u: int, v: int, plain=False) -> float:
    return _load(plain).orc_pair_coin(seed, u, v)


def K_of_c(c, d, T, plain=False) -> float:
    """The scale K of the model for the c of Eq. 1: c^T (T > 0) or c^d (T = 0)."""
    return _load(plain).orc_girg_K_of_c(c, d, T)


def c_of_K(K, d, T) -> float:
    """The c of Eq. 1 for a scale K (0 or inf where it leaves the range of doubles)."""
    e = math.log(K) / (T if T > 0.0 else d)
    return 0.0 if e < -745.0 else (math.inf if e > 709.0 else math.exp(e))


def _scale(c, d, T, K, plain=False):
    return K if K is not None else K_of_c(c, d, T, plain=plain)


def girg_p(d, T, c, W, wu, wv, D, K=None, plain=False) -> float:
    """Eq. 1, p = min{1, (K q / r^d)^(1/T)} with K = c^T (c ignored if K is given)."""
    return _load(plain).orc_girg_p(d, T, _scale(c, d, T, K, plain), W, wu, wv, D)


def girg_thresh_edge(d, c, W, wu, wv, D, K=None, plain=False) -> bool:
    """Threshold variant: r^d <= K w_u w_v / W with K = c^d."""
    return bool(_load(plain).orc_girg_thresh_edge(d, _scale(c, d, 0.0, K, plain), W, wu, wv, D))


def hrg_coshd(ru, rv, D, plain=False) -> float:
    return _load(plain).orc_hrg_coshd(ru, rv, D)


def hrg_p(T, R, ru, rv, D, plain=False) -> float:
    return _load(plain).orc_hrg_p(T, R, ru, rv, D)


def hrg_weight(r, R, plain=False) -> float:
    return _load(plain).orc_hrg_weight(r, R)


# ---------------------------------------------------------------- model inputs

def girg_points(n: int, d: int, beta: float, w_min: float, seed: int, plain=False):
    """Weights (n,) float64 and positions (n, d) uint32 of the generated GIRG."""
    w = np.zeros(n, dtype=np.float64)
    X = np.zeros((n, d), dtype=np.uint32)
    _load(plain).orc_girg_points(n, d, beta, w_min, seed, _ptr(w), _ptr(X))
    return w, X


def hrg_points(n: int, alpha: float, R: float, seed: int, plain=False):
    """Radii (n,) float64 and angular fixed-point coordinates (n,) uint32."""
    r = np.zeros(n, dtype=np.float64)
    X = np.zeros(n, dtype=np.uint32)
    _load(plain).orc_hrg_points(n, alpha, R, seed, _ptr(r), _ptr(X))
    return r, X


# ---------------------------------------------------------------- samplers

def _edges_array(cap):
    return np.zeros((max(cap, 1), 2), dtype=np.uint32)


def girg_allpairs(X, w, W, T, c, seed, cap=None, K=None, plain=False):
    """Oracle 1: (m, 2) uint32 edges (u < v) of the quadratic generator."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, d = X.shape
    K = _scale(c, d, T, K, plain)
    if cap is None:
        cap = 1 << 16
    while True:
        e = _edges_array(cap)
        m = _load(plain).orc_girg_allpairs(n, d, _ptr(X), _ptr(w), W, T, K, seed, _ptr(e), cap)
        if m <= cap:
            return e[:m].copy()
        cap = m


def hrg_allpairs(X, r, R, T, seed, cap=None, plain=False):
    X = np.ascontiguousarray(X, dtype=np.uint32)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = len(X)
    if cap is None:
        cap = 1 << 16
    while True:
        e = _edges_array(cap)
        m = _load(plain).orc_hrg_allpairs(n, _ptr(X), _ptr(r), R, T, seed, _ptr(e), cap)
        if m <= cap:
            return e[:m].copy()
        cap = m


class CellPairResult:
    """Edges, statistics, sorted order, tables and (optionally) items of oracle 2."""

    def __init__(self, edges, stats, order, itab, wtab, items):
        self.edges = edges
        self.stats = dict(zip(STAT_NAMES, (int(s) for s in stats[:8])))
        self.visited_neighbour = stats[8:8 + 33].copy()
        self.visited_distant = stats[8 + 33:8 + 66].copy()
        self.visited_self = stats[8 + 66:8 + 99].copy()
        self.order = order
        L = int(itab[0])
        self.L = L
        self.level_cap = int(itab[1])
        self.max_level = int(itab[2])
        self.I = itab[3:3 + L].astype(np.int64)
        self.CL = itab[3 + MAXL:3 + MAXL + MAXL * MAXL].reshape(MAXL, MAXL)[:L, :L].astype(
            np.int64)
        self.wmax = wtab[:L].copy()
        self.layer_count = wtab[MAXL:MAXL + L].astype(np.int64)
        self.items = items


ITEM_FIELDS = ("type", "level", "A", "B", "i", "j", "a_lo", "a_hi", "b_lo", "b_hi", "tri",
               "pbar")


def _items_to_records(raw, k):
    raw = raw[:k]
    out = {}
    for col, name in enumerate(ITEM_FIELDS):
        if name == "pbar":
            out[name] = raw[:, col].copy().view(np.float64)
        else:
            out[name] = raw[:, col].copy()
    return out


def girg_cellpairs(X, w, w_min, W, T, c, seed, cap=None, want_items=False, skip_sampling=False,
                   items_cap=None, level_cap=0, K=None, plain=False):
    """Oracle 2 for GIRGs (Algorithm 1 with App. B.1)."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, d = X.shape
    K = _scale(c, d, T, K, plain)
    if cap is None:
        cap = 1 << 16
    while True:
        e = _edges_array(cap)
        stats = np.zeros(8 + 99, dtype=np.int64)
        order = np.zeros(max(n, 1), dtype=np.int64)
        itab = np.zeros(3 + MAXL + MAXL * MAXL, dtype=np.int32)
        wtab = np.zeros(2 * MAXL, dtype=np.float64)
        nitems = np.zeros(1, dtype=np.int64)
        icap = items_cap if items_cap is not None else (1 << 20)
        items = np.zeros((icap if want_items else 1, 12), dtype=np.int64)
        m = _load(plain).orc_girg_cellpairs(
            n, d, _ptr(X), _ptr(w), w_min, W, T, K, seed, _ptr(e), cap, _ptr(stats),
            _ptr(order), _ptr(itab), _ptr(wtab), _ptr(items) if want_items else None,
            icap if want_items else 0, _ptr(nitems), 1 if skip_sampling else 0, level_cap)
        if m < 0:
            raise RuntimeError("a type-II stream needs more than 2^32 chunks")
        if want_items and nitems[0] > icap:
            items_cap = int(nitems[0])
            continue
        if m <= cap:
            recs = _items_to_records(items, int(nitems[0])) if want_items else None
            return CellPairResult(e[:m].copy(), stats, order[:n], itab, wtab, recs)
        cap = m


def hrg_cellpairs(X, r, R, T, seed, cap=None, want_items=False, skip_sampling=False,
                  items_cap=None, level_cap=0, plain=False):
    """Oracle 2 for HRGs through the HRG -> GIRG mapping of Sec. 2.3."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = len(X)
    if cap is None:
        cap = 1 << 16
    while True:
        e = _edges_array(cap)
        stats = np.zeros(8 + 99, dtype=np.int64)
        order = np.zeros(max(n, 1), dtype=np.int64)
        itab = np.zeros(3 + MAXL + MAXL * MAXL, dtype=np.int32)
        wtab = np.zeros(2 * MAXL, dtype=np.float64)
        nitems = np.zeros(1, dtype=np.int64)
        icap = items_cap if items_cap is not None else (1 << 20)
        items = np.zeros((icap if want_items else 1, 12), dtype=np.int64)
        m = _load(plain).orc_hrg_cellpairs(
            n, _ptr(X), _ptr(r), R, T, seed, _ptr(e), cap, _ptr(stats), _ptr(order),
            _ptr(itab), _ptr(wtab), _ptr(items) if want_items else None,
            icap if want_items else 0, _ptr(nitems), 1 if skip_sampling else 0, level_cap)
        if m < 0:
            raise RuntimeError("a type-II stream needs more than 2^32 chunks")
        if want_items and nitems[0] > icap:
            items_cap = int(nitems[0])
            continue
        if m <= cap:
            recs = _items_to_records(items, int(nitems[0])) if want_items else None
            return CellPairResult(e[:m].copy(), stats, order[:n], itab, wtab, recs)
        cap = m


# ---------------------------------------------------------------- degree / c

def girg_avg_degree(c, w, d, T, W=None, K=None, plain=False):
    """Expected average degree f of App. B.2 for the given weights at c (or scale K)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    if W is None:
        W = exact_sum(w, plain=plain)
    return _load(plain).orc_girg_avg_degree(_scale(c, d, T, K, plain), len(w), d, T, _ptr(w), W)


def girg_solve_K(target, w, d, T, W=None, plain=False):
    """The scale K (c^T, or c^d at T = 0) whose expected average degree is ``target``."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    if W is None:
        W = exact_sum(w, plain=plain)
    return _load(plain).orc_girg_solve_K(target, len(w), d, T, _ptr(w), W)


def girg_solve_c(target, w, d, T, W=None, plain=False):
    """The c of Eq. 1 whose expected average degree is ``target`` (App. B.2)."""
    return c_of_K(girg_solve_K(target, w, d, T, W, plain=plain), d, T)


def hrg_avg_degree(n, alpha, T, R, plain=False):
    """Expected average degree of an HRG (radius R), by quadrature of its definition."""
    return _load(plain).orc_hrg_avg_degree(n, alpha, T, R)


def hrg_solve_R(n, alpha, T, target, plain=False):
    """The disk radius R with expected average degree ``target`` (bisection)."""
    return _load(plain).orc_hrg_solve_R(n, alpha, T, target)


def girg_thresh_neighbors(X, w, W, K, us, cap=None, plain=False):
    """Threshold model by brute force: every (u, v), u in ``us``, v != u, with
    r^d <= K w_u w_v / W, as an (m, 2) int64 array."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    us = np.ascontiguousarray(us, dtype=np.int64)
    n, d = X.shape
    cap = cap or 1 << 16
    while True:
        out = np.zeros((cap, 2), dtype=np.int64)
        m = _load(plain).orc_girg_thresh_neighbors(n, d, _ptr(X), _ptr(w), W, K, _ptr(us), len(us),
                                              _ptr(out), cap)
        if m <= cap:
            return out[:m]
        cap = m


class audit:
    """Decision audit of the samplers in the selected build (a context manager):
    counts every decision taken inside the ``with`` block and records the near ones,
    whose two sides are within a relative ``eps`` of each other.  ``records`` is an
    (k, 3) int64 array of (kind, a, b): kind 1 per-pair coin, 2 type-II acceptance,
    3 threshold test (a < b vertex ids), 4 geometric jump near an integer (a = cell A,
    b = stream word << 32 | chunk); ``count`` the number of near decisions (records
    holds at most ``cap`` of them) and ``decisions`` the number of all decisions."""

    def __init__(self, eps=1e-12, cap=1 << 16, plain=False):
        self.eps, self.cap, self.plain = eps, cap, plain
        self._buf = np.zeros((cap, 3), dtype=np.int64)
        self.records = self._buf[:0]
        self.count = 0
        self.decisions = 0

    def __enter__(self):
        _load(self.plain).orc_audit_begin(self.eps, _ptr(self._buf), self.cap)
        return self

    def __exit__(self, *exc):
        dec = np.zeros(1, dtype=np.int64)
        self.count = int(_load(self.plain).orc_audit_end(_ptr(dec)))
        self.decisions = int(dec[0])
        self.records = self._buf[:min(self.count, self.cap)].copy()
        return False

    def pairs(self, kinds=(1, 2, 3)) -> set:
        """The recorded vertex pairs (keys u 2^32 + v, u < v) of the given kinds."""
        r = self.records[np.isin(self.records[:, 0], kinds)]
        return set((r[:, 1] * (1 << 32) + r[:, 2]).tolist())


def splitmix64_finalize(z):
    """The output function of splitmix64 (Steele, Lea, Flood, OOPSLA 2014) on uint64."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def edge_checksum(edges) -> int:
    """Order-independent checksum of an edge list: the sum mod 2^64 of
    splitmix64_finalize(u 2^32 + v) over the edges, u < v."""
    e = np.asarray(edges, dtype=np.uint64).reshape(-1, 2)
    if len(e) == 0:
        return 0
    key = (np.minimum(e[:, 0], e[:, 1]) << np.uint64(32)) | np.maximum(e[:, 0], e[:, 1])
    with np.errstate(over="ignore"):
        return int(np.sum(splitmix64_finalize(key), dtype=np.uint64))


def edge_set(edges) -> set:
    """Set of (u, v) tuples with u < v from an (m, 2) array."""
    e = np.asarray(edges, dtype=np.int64)
    if len(e) == 0:
        return set()
    key = np.minimum(e[:, 0], e[:, 1]) * (1 << 32) + np.maximum(e[:, 0], e[:, 1])
    return set(key.tolist())
