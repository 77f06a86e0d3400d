"""Pins of the oracle's primitives against sources other than the oracle itself.

* Philox4x32-10 against the published known-answer vectors (tests/golden) and
  against an independent implementation (Triton's interpreter, when present).
* The deterministic elementary functions against mpmath at 60 digits.
* The exact sum against ``math.fsum`` (exactly rounded by construction).
* The Morton layout against the worked example of Sec. 4.2.
* The visited cell-pair counts against Fig. 5b and App. B.5.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = O.philox(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_philox_matches_independent_implementation():
    """Triton's Philox (same published constants) run on the CPU interpreter."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    code = r"""
import os
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out, seed, N: tl.constexpr):
    off = tl.arange(0, N)
    a, b, c, d = tl.randint4x(seed, off)
    tl.store(out + off * 4 + 0, a); tl.store(out + off * 4 + 1, b)
    tl.store(out + off * 4 + 2, c); tl.store(out + off * 4 + 3, d)
out = torch.zeros(64, dtype=torch.int32)
k[(1,)](out, 123456789, N=16)
print(" ".join(str(x & 0xffffffff) for x in out.tolist()))
"""
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-200:])
    words = [int(t) for t in res.stdout.split()]
    for i in range(16):
        # triton: counter = (offset, 0, 0, 0), key = (seed_lo, seed_hi)
        out = O.philox([i, 0, 0, 0], [123456789, 0])
        assert [int(x) for x in out] == words[4 * i:4 * i + 4]


def test_uniform_grid():
    assert O.uniform(0, 0) == 2.0 ** -53
    assert O.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    u = O.uniform(0x12345678, 0x9ABCDEF0)
    assert 0.0 < u < 1.0
    bits = (0x9ABCDEF0 << 32) | 0x12345678
    assert u == (2 * (bits >> 12) + 1) / 2.0 ** 53


mp = pytest.importorskip("mpmath")


def _ulp_err(got, ref):
    ref_f = float(ref)
    if ref_f == 0.0:
        return abs(got) / 5e-324
    return abs(mp.mpf(got) - ref) / mp.mpf(math.ulp(ref_f))


def test_det_log_exp_against_mpmath():
    mp.mp.dps = 60
    rng = np.random.default_rng(5)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(0.5, 2.0, 2000),
                         1.0 + rng.uniform(-1e-6, 1e-6, 500), [5e-324, 1e-310, 2.2250738585072014e-308]])
    worst = 0
    for x in xs:
        worst = max(worst, _ulp_err(O.det_log(x), mp.log(mp.mpf(x))))
    # fixed point to about 2^-60 relative, rounded once: within 0.5 ulp plus a little
    assert worst <= 0.55, worst
    ys = np.concatenate([rng.uniform(-740, 709, 3000), rng.uniform(-1, 1, 2000)])
    worst = 0
    for y in ys:
        worst = max(worst, _ulp_err(O.det_exp(y), mp.exp(mp.mpf(y))))
    # rounded once, except below 2^-1022 where the scaling rounds a second time
    assert worst <= 1.0, worst
    assert O.det_exp(0.0) == 1.0 and O.det_log(1.0) == 0.0
    assert O.det_exp(800.0) == math.inf and O.det_exp(-800.0) == 0.0
    assert O.det_log(0.0) == -math.inf


def test_det_log_exp_monotone_and_exact_points():
    """Monotone across every table boundary (a wrong table entry or reduction breaks this),
    exact at 1 and 0, and correctly rounded at powers of two and at the table points."""
    mp.mp.dps = 60
    rng = np.random.default_rng(8)
    xs = np.sort(np.concatenate([rng.uniform(0.70, 1.42, 200000),
                                 np.exp(rng.uniform(-700, 700, 20000))]))
    logs = np.array([O.det_log(float(x)) for x in xs])
    assert np.all(np.diff(logs) >= 0)
    ys = np.sort(np.concatenate([rng.uniform(-0.02, 0.02, 100000), rng.uniform(-740, 709, 50000)]))
    exps = np.array([O.det_exp(float(y)) for y in ys])
    assert np.all(np.diff(exps) >= 0)
    assert O.det_log(1.0) == 0.0 and O.det_exp(0.0) == 1.0
    for k in range(-1074, 1024, 7):
        x = math.ldexp(1.0, k)
        assert O.det_log(x) == float(mp.mpf(k) * mp.log(2)), k
    for j in range(45, 92):
        x = j / 64.0
        assert O.det_log(x) == float(mp.log(mp.mpf(x))), j
    for j in range(64):  # 2^(j/64) at the reduction points k ln2/64 (up to the rounding of x)
        x = j * math.log(2) / 64
        assert _ulp_err(O.det_exp(x), mp.exp(mp.mpf(x))) <= 0.51, j


def test_det_log_exp_dense_at_table_boundaries_against_mpmath():
    """The fixed-point ln and exp are the same method as the CUDA library's (so that both
    take identical decisions); this sweep pins that method itself against 60-digit
    arithmetic where a wrong table entry or reduction would show first: significands
    within 64 ulps of every switch of the table index j = round(64 m), and arguments
    within 64 ulps of every switch of the reduction k = round(64 x / ln 2)."""
    mp.mp.dps = 60
    worst = 0
    offs = list(range(-64, 65, 4))
    for j in range(45, 92):
        for e in (-600, -3, 0, 1, 40, 700):
            edge = math.ldexp((j + 0.5) / 64.0, e)
            for k in offs:
                x = edge + k * math.ulp(edge)
                if x <= 0:
                    continue
                worst = max(worst, _ulp_err(O.det_log(x), mp.log(mp.mpf(x))))
    assert worst <= 0.55, worst
    worst = 0
    ln2_64 = mp.log(2) / 64
    for kk in list(range(-40, 41)) + list(range(-60000, 60001, 1499)):
        edge = float((kk - mp.mpf(0.5)) * ln2_64)
        for k in offs:
            y = edge + k * math.ulp(edge if edge else 1e-300)
            ref = mp.exp(mp.mpf(y))
            if float(ref) < 2.2250738585072014e-308:
                continue
            worst = max(worst, _ulp_err(O.det_exp(y), ref))
    assert worst <= 0.55, worst


def test_det_log1p_and_pow_against_mpmath():
    mp.mp.dps = 60
    rng = np.random.default_rng(6)
    worst = 0
    for x in np.concatenate([-np.exp(rng.uniform(-40, math.log(0.999), 3000)),
                             rng.uniform(-0.3, 0.3, 1000)]):
        worst = max(worst, _ulp_err(O.det_log1p(x), mp.log1p(mp.mpf(x))))
    # for x < -1/4 the rounding of 1 + x adds up to about 2 ulp
    assert worst <= 4.0, worst
    # pow = exp(y ln x): relative error grows with |y ln x|, bounded by 2^-52 (|y ln x| + 4)
    for _ in range(3000):
        x = float(np.exp(rng.uniform(-60, 60)))
        y = float(rng.uniform(-10, 10))
        ref = mp.power(mp.mpf(x), mp.mpf(y))
        if float(ref) == 0.0 or math.isinf(float(ref)):
            continue
        rel = abs(mp.mpf(O.det_pow(x, y)) - ref) / ref
        assert rel <= 2.0 ** -52 * (abs(y * math.log(x)) + 4), (x, y, rel)


def test_det_sinpi_acosh_against_mpmath():
    mp.mp.dps = 60
    rng = np.random.default_rng(7)
    worst = 0
    for x in np.concatenate([rng.uniform(0, 0.5, 4000), np.exp(rng.uniform(-40, -2, 1000)),
                             [0.25, 0.5, 0.0]]):
        worst = max(worst, _ulp_err(O.det_sinpi(x), mp.sin(mp.pi * mp.mpf(x))))
    assert worst <= 3.0, worst
    for z in np.exp(rng.uniform(0.01, 60, 2000)):
        ref = mp.acosh(mp.mpf(z))
        assert abs(mp.mpf(O.det_acosh(z)) - ref) / ref < 1e-15


def test_exact_sum_matches_fsum():
    rng = np.random.default_rng(8)
    for scale in (1.0, 1e6, 1e-3):
        w = scale * (1.0 + rng.pareto(1.2, 100000))
        assert O.exact_sum(w) == math.fsum(w)
    w = np.array([1.0, 2.0 ** 60, 1.0, -0.0 + 3.0])
    assert O.exact_sum(w) == math.fsum(w)
    # ties to even
    w = np.array([2.0 ** 53, 1.0])
    assert O.exact_sum(w) == math.fsum(w) == 2.0 ** 53
    w = np.array([2.0 ** 53, 1.0, 1.0])
    assert O.exact_sum(w) == 2.0 ** 53 + 2


def test_morton_worked_example():
    """Sec. 4.2: 4-bit a = a3a2a1a0, b = b3b2b1b0 -> a3 b3 a2 b2 a1 b1 a0 b0."""
    a, b = 0b1010, 0b0110
    x = [a << 28, b << 28]
    code = O.morton(x, 2, 4)
    expect = 0
    for bit in range(3, -1, -1):
        expect = (expect << 1) | ((a >> bit) & 1)
        expect = (expect << 1) | ((b >> bit) & 1)
    assert code == expect == 0b10011100
    # the descendants of a level-1 cell are consecutive on level 2 (Sec. 3.4 (I))
    for cell1 in range(4):
        kids = sorted(O.morton([((cell1 >> 1) << 31) | (c0 << 30), ((cell1 & 1) << 31) | (c1 << 30)],
                               2, 2) for c0 in (0, 1) for c1 in (0, 1))
        assert kids == list(range(4 * cell1, 4 * cell1 + 4))


def test_level_cap_and_chunk_log():
    # T = 0: (bitlen(n) + 4) / d, at most 32 / d
    assert O.level_cap(10000, 1, 0.0) == 18
    assert O.level_cap(1_000_000, 2, 0.0) == 12
    assert O.level_cap(2 ** 24, 4, 0.0) == 7
    assert O.level_cap(2 ** 30, 1, 0.0) == 32
    # T > 0: floor(log2(n)/d - 1/2) with log2 n = bitlen(n) - 1, about 2^(d/2) vertices
    # per cell of the deepest level
    assert O.level_cap(2 ** 24, 1, 0.7) == 23
    assert O.level_cap(2 ** 24, 2, 0.7) == 11
    assert O.level_cap(2 ** 24, 3, 0.7) == 7
    assert O.level_cap(2 ** 24, 4, 0.7) == 5
    assert O.level_cap(1_000_000, 2, 0.5) == 9
    assert O.level_cap(10, 4, 0.5) == 1
    for p in (0.75, 0.5, 1e-3, 3e-9):
        k = O.chunk_log(p)
        assert 4 <= p * 2 ** k < 8
    assert O.chunk_log(1.0) == 3
    assert O.chunk_log(1e-9) == O.chunk_log(1e-30) == 31  # clamped: chunks of 2^31


def _visit_counts(d, depth):
    """Visited cell pairs of the recursion for a graph whose deepest level is
    ``depth`` (one weight bucket, c tuned so that CL = depth)."""
    n = 2 ** 10
    w = np.ones(n)
    X = np.zeros((n, d), dtype=np.uint32)
    rng = np.random.default_rng(1)
    X[:] = rng.integers(0, 2 ** 32, size=(n, d), dtype=np.uint64).astype(np.uint32)
    W = float(n)
    # threshold variant: kappa = c (1/W)^(1/d); choose kappa = 0.75 * 2^-depth
    c = 0.75 * 2.0 ** -depth / (1.0 / W) ** (1.0 / d)
    res = O.girg_cellpairs(X, w, 1.0, W, 0.0, c, 1, skip_sampling=True, level_cap=depth + 1)
    assert res.max_level == depth
    return res


def test_visited_cell_pairs_match_fig5b_d1():
    """Fig. 5b: 8 neighbouring pairs on level 2, 12 distant pairs on level 3."""
    res = _visit_counts(1, 6)
    assert res.visited_neighbour[2] == 8
    assert res.visited_distant[3] == 12
    # App. B.5 (d = 1, l > 2): 2^l heavy (A, A), 2^l light (A, A+1), 3 2^(l-1) distant
    for lvl in range(3, 7):
        assert res.visited_self[lvl] == 2 ** lvl
        assert res.visited_neighbour[lvl] - res.visited_self[lvl] == 2 ** lvl
        assert res.visited_distant[lvl] == 3 * 2 ** (lvl - 1)


def test_visited_cell_pairs_heavy_tasks_d2():
    """App. B.5: the number of heavy tasks in d dimensions is 2^(l d)."""
    res = _visit_counts(2, 4)
    for lvl in range(0, 5):
        assert res.visited_self[lvl] == 2 ** (2 * lvl)
    # all cells are neighbours on levels 0 and 1 (torus)
    assert res.visited_distant[0] == 0 and res.visited_distant[1] == 0
    # level 1: 4 cells -> 4 * 5 / 2 unordered pairs incl. self
    assert res.visited_neighbour[1] == 10


def test_splitmix64_finalizer_known_outputs():
    """The edge checksum's mixing function against the first outputs of splitmix64."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if ln.strip() and not ln.startswith("#")]
    for k, state, out in rows:
        assert int(state, 16) == (int(k) * 0x9E3779B97F4A7C15) % (1 << 64)
        assert int(O.splitmix64_finalize(np.uint64(int(state, 16)))) == int(out, 16)


def test_edge_checksum_is_order_independent():
    rng = np.random.default_rng(3)
    e = rng.integers(0, 1 << 31, size=(1000, 2))
    assert O.edge_checksum(e) == O.edge_checksum(e[::-1]) == O.edge_checksum(e[:, ::-1])
    assert O.edge_checksum(e[:999]) != O.edge_checksum(e)


def test_layer_boundaries():
    """Sec. 3.1 buckets: weights in [w_min 2^i, w_min 2^(i+1)) form bucket i.  Checked at
    every boundary, one ulp on either side, against the exact binary logarithm of the
    rounded quotient (Fraction arithmetic), and clamped below at 0."""
    from fractions import Fraction

    def exact(w, w_min):
        q = Fraction(w / w_min)  # the FP64 quotient, exactly
        i = 0
        while q >= 2:
            q /= 2
            i += 1
        return min(i, 63)

    for w_min in (1.0, 0.75, 1.5, 3.0e-7, 12345.678):
        for i in range(0, 62):
            b = w_min * 2.0 ** i
            for w in (b, math.nextafter(b, 0.0), math.nextafter(b, math.inf)):
                if w >= w_min:
                    assert O.layer_of(w, w_min) == exact(w, w_min), (w_min, i, w)
        assert O.layer_of(w_min, w_min) == 0
        assert O.layer_of(math.nextafter(w_min, 0.0), w_min) == 0
