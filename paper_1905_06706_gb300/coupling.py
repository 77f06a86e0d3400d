"""HRGs against GIRGs (Sec. 5, "Difference between HRGs and GIRGs"; Sec. 2.3).

For a threshold HRG (T = 0), the GIRG on the same vertices through the mapping of
Sec. 2.3 (weights e^((R - r)/2), angles on the 1-dimensional torus) connects u, v iff
r_uv <= K w_u w_v / W; the graph only grows with the scale K.  The experiment finds
the largest K whose GIRG is a subgraph of the HRG (its average degree is d_girg) and
the smallest K whose GIRG is a supergraph (D_girg), each by bisection on log K with
exact edge-set differences, and the numbers of missing (HRG minus GIRG) and
additional (GIRG minus HRG) edges along a grid of scales.  Both graphs are generated
by the library's kernels; the set differences are sorted-key lookups on the device.
"""
from __future__ import annotations

import math

from . import (GIRG_E_CAPACITY, GIRG_OK, PRECISION_FP32, GirgError, _torch,
               girg_generate_from_points, hrg_generate, hrg_girg_points)


def _keys(torch, e, m, n):
    e = e[:m].to(torch.int64)
    return torch.sort(e[:, 0] * n + e[:, 1]).values


def _generate(torch, fn, cap):
    while True:
        ed = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
        r = fn(ed)
        if r.status == GIRG_OK:
            return ed, r.num_edges
        if r.status != GIRG_E_CAPACITY:
            raise GirgError(r.status, "generation")
        cap = r.num_edges + 1024


class Coupling:
    """One threshold HRG and the GIRGs on its vertices."""

    def __init__(self, n, alpha, R, seed=1):
        torch = self.torch = _torch()
        self.n = n
        eh, mh = _generate(torch, lambda ed: hrg_generate(ed, n=n, alpha=alpha, T=0.0, R=R,
                                                          seed=seed), n * 16)
        self.hrg_edges = mh
        self.kh = _keys(torch, eh, mh, n)
        del eh
        self.w, self.X = hrg_girg_points(n, alpha, R, seed)

    def compare(self, K):
        """(GIRG edge count, missing, additional) of the GIRG with scale K."""
        torch = self.torch
        cap = max(1024, int(2 * self.hrg_edges))
        eg, mg = _generate(torch, lambda ed: girg_generate_from_points(
            ed, self.X, self.w, T=0.0, c=K, seed=0, precision=PRECISION_FP32), cap)
        kg = _keys(torch, eg, mg, self.n)
        del eg
        if mg == 0 or self.hrg_edges == 0:
            common = 0
        else:
            pos = torch.searchsorted(self.kh, kg).clamp_(max=self.hrg_edges - 1)
            common = int((self.kh[pos] == kg).sum())
        return mg, self.hrg_edges - common, mg - common

    def _bisect(self, ok, K0, rel_tol):
        """Largest K with ok(K) (ok true for small K, false for large)."""
        lo = hi = K0
        if ok(K0):
            hi = K0 * 2.0
            while ok(hi):
                lo, hi = hi, hi * 2.0
        else:
            lo = K0 / 2.0
            while not ok(lo):
                lo, hi = lo / 2.0, lo
        while hi - lo > rel_tol * hi:
            mid = math.sqrt(lo * hi)
            if ok(mid):
                lo = mid
            else:
                hi = mid
        return lo, hi

    def run(self, grid=(), rel_tol=1e-6):
        n = self.n
        d_hrg = 2.0 * self.hrg_edges / n
        # start near the scale whose GIRG has the HRG's degree: K ~ d W / (2 n) (d = 1)
        K0 = d_hrg * float(self.w.sum()) / (2.0 * n)
        k_sub, _ = self._bisect(lambda K: self.compare(K)[2] == 0, K0, rel_tol)
        _, k_sup = self._bisect(lambda K: self.compare(K)[1] > 0, K0, rel_tol)
        m_sub = self.compare(k_sub)[0]
        m_sup = self.compare(k_sup)[0]
        curve = []
        for K in grid:
            mg, miss, add = self.compare(K)
            curve.append({"K": K, "girg_degree": 2.0 * mg / n, "missing": miss,
                          "additional": add})
        return {"n": n, "hrg_edges": self.hrg_edges, "d_hrg": d_hrg,
                "K_sub": k_sub, "d_girg": 2.0 * m_sub / n,
                "K_super": k_sup, "D_girg": 2.0 * m_sup / n, "curve": curve}


def hrg_girg_coupling(n, alpha, R, seed=1, grid=(), rel_tol=1e-6) -> dict:
    """d_hrg, d_girg, D_girg (with their scales) and the missing / additional edge curve
    for the threshold HRG with n vertices, dispersion alpha, radius R and seed."""
    return Coupling(n, alpha, R, seed).run(grid, rel_tol)
