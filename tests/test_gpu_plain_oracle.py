"""The CUDA path against the plain build of the oracle (the C library's log, exp, log1p,
pow, sin and acosh; no arithmetic shared with the library beyond IEEE +, -, *, /).

The sampler is exact (Sec. 3.2: no approximation), so with the same coins the two
graphs differ only where a decision is so close to its threshold that the two sides'
different roundings of Eq. 1, p_T(d) (Sec. 2.2) or the jump ln U / ln(1 - pbar) flip
it.  The bar: at most 1e-9 of all decisions flipped, and every flipped pair recorded by
the oracle's decision audit as within a relative 1e-12 of its threshold.  Each test
reports the number of decisions, of near decisions and of flips.

GIRG inputs are the plain oracle's points, passed to the library through
girg_generate_from_points with the plain oracle's c (that entry point takes the smallest
weight as the bucket unit, and so does the oracle here); the HRG draws its points on
each side (radii through acosh and exp, so they differ by a few ulps).
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_06706_gb300 as gg  # noqa: E402

EPS = 1e-12          # how close to its threshold a flipped decision may be
MAX_FLIP_SHARE = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gg.load()


def _set(ed, m):
    e = ed[:m].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    assert np.all(e[:, 0] < e[:, 1])
    s = set((e[:, 0] * (1 << 32) + e[:, 1]).tolist())
    assert len(s) == m
    return s


def _check(got: set, ref_edges, aud: O.audit, what: str):
    ref = O.edge_set(ref_edges)
    flips = got ^ ref
    print(f"{what}: {aud.decisions} decisions, {aud.count} within {EPS:g} of the "
          f"threshold, {len(flips)} flipped")
    assert aud.count <= aud.cap
    assert flips <= aud.pairs(), f"{what}: a flipped pair is not near its threshold"
    assert len(flips) <= MAX_FLIP_SHARE * aud.decisions, what
    assert abs(len(got) - len(ref)) <= len(flips)


def _girg_case(n, d, beta, T, deg, seed, eb=4):
    w, X = O.girg_points(n, d, beta, 1.0, seed, plain=True)
    W = O.exact_sum(w, plain=True)
    c = O.girg_solve_c(deg, w, d, T, W, plain=True)
    with O.audit(EPS, plain=True) as aud:
        ref = O.girg_cellpairs(X, w, float(w.min()), W, T, c, seed, cap=int(n * deg * 1.5),
                               plain=True)
    Xg = torch.from_numpy(np.ascontiguousarray(X.T).view(np.int32)).cuda()
    wg = torch.from_numpy(w).cuda()
    ed = torch.empty((int(n * deg * 1.5), 2), dtype=torch.int32 if eb == 4 else torch.int64,
                     device="cuda")
    return Xg, wg, W, c, ref, aud, ed


@pytest.mark.parametrize("precision", [0, 1])
def test_benchmark_shape_against_plain_oracle(precision):
    """d = 2, beta = 2.5, T = 0.5, average degree 10 (the benchmark's parameters) at
    n = 2 10^5, both precision modes of the library."""
    n, d, T, seed = 200_000, 2, 0.5, 1
    Xg, wg, W, c, ref, aud, ed = _girg_case(n, d, 2.5, T, 10.0, seed)
    r = gg.girg_generate_from_points(ed, Xg, wg, T=T, c=c, seed=seed, precision=precision)
    assert r.status == gg.GIRG_OK, gg.status_string(r.status)
    _check(_set(ed, r.num_edges), ref.edges, aud, f"girg d=2 T=0.5 fp{64 if precision else 32}")


SWEEP_N = {1: 1 << 17, 2: 1 << 16, 3: 1 << 15, 4: 1 << 13}


@pytest.mark.parametrize("d,T", [(1, 0.7), (2, 0.7), (3, 0.7), (4, 0.7), (2, 0.0)])
def test_dimension_sweep_against_plain_oracle(d, T):
    """The dimension sweep's parameters (beta = 2.2, average degree 16, int64 edges) at
    reduced n; T = 0.7 evaluates p = x^(1/T) through exp and log on both sides."""
    n, seed = SWEEP_N[d], 3
    Xg, wg, W, c, ref, aud, ed = _girg_case(n, d, 2.2, T, 16.0, seed, eb=8)
    r = gg.girg_generate_from_points(ed, Xg, wg, T=T, c=c, seed=seed)
    assert r.status == gg.GIRG_OK, gg.status_string(r.status)
    _check(_set(ed, r.num_edges), ref.edges, aud, f"girg d={d} T={T}")


@pytest.mark.parametrize("T", [0.5, 0.0])
def test_hrg_against_plain_oracle(T):
    n, alpha, seed = 200_000, 0.75, 2
    R = O.hrg_solve_R(n, alpha, T, 10.0, plain=True)
    rr, X = O.hrg_points(n, alpha, R, seed, plain=True)
    with O.audit(EPS, plain=True) as aud:
        ref = O.hrg_cellpairs(X, rr, R, T, seed, cap=n * 16, plain=True)
    ed = torch.empty((n * 16, 2), dtype=torch.int32, device="cuda")
    r = gg.hrg_generate(ed, n=n, alpha=alpha, T=T, R=R, seed=seed)
    assert r.status == gg.GIRG_OK, gg.status_string(r.status)
    _check(_set(ed, r.num_edges), ref.edges, aud, f"hrg T={T}")


@pytest.mark.parametrize("precision", [0, 1])
def test_allpairs_config_against_plain_oracle(precision):
    """d = 1, n = 10^4, beta = 2.5, T = 0.5, average degree 10, seed 1: the GPU all-pairs
    kernel against the plain quadratic generator, the GPU cell-pair sampler against the
    plain cell-pair sampler (the two samplers draw type-II pairs from different coins)."""
    n, d, T, seed = 10_000, 1, 0.5, 1
    w, X = O.girg_points(n, d, 2.5, 1.0, seed, plain=True)
    W = O.exact_sum(w, plain=True)
    c = O.girg_solve_c(10.0, w, d, T, W, plain=True)
    with O.audit(EPS, plain=True) as aud:
        ref = O.girg_allpairs(X, w, W, T, c, seed, plain=True)
    assert aud.decisions == n * (n - 1) // 2
    Xg = torch.from_numpy(np.ascontiguousarray(X.T).view(np.int32)).cuda()
    wg = torch.from_numpy(w).cuda()
    ed = torch.empty((n * 16, 2), dtype=torch.int32, device="cuda")
    r = gg.girg_allpairs(ed, Xg, wg, W=W, T=T, c=c, seed=seed, precision=precision)
    assert r.status == gg.GIRG_OK
    _check(_set(ed, r.num_edges), ref, aud, "all pairs d=1 T=0.5")
    with O.audit(EPS, plain=True) as aud2:
        ref2 = O.girg_cellpairs(X, w, float(w.min()), W, T, c, seed, cap=n * 16, plain=True)
    r = gg.girg_generate_from_points(ed, Xg, wg, T=T, c=c, seed=seed, precision=precision)
    assert r.status == gg.GIRG_OK
    _check(_set(ed, r.num_edges), ref2.edges, aud2, "cell pairs d=1 T=0.5")
