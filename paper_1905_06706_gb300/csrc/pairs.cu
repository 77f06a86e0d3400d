// Edge sampling: the cell pairs of Algorithm 1 (Sec. 3.3) with the
// double-counting rules of App. B.1, all-pairs tests on neighbouring cells
// (type I), geometric jumps with rejection on distant cells (type II, Sec. 3.2),
// and warp-aggregated compaction of the edges.
//
// Instead of recursing from the root pair, the device enumerates "rows"
// (bucket i, level l, non-empty cell A of V_i at level l).  A warp takes a row
// and its lanes take the (bucket j, cell B) combinations that Algorithm 1
// processes with A: the neighbours B of A when CL(i,j) = l (type I) and the
// cells B that are distant from A but have neighbouring parents when
// CL(i,j) >= l (type II), for buckets j >= i; for j = i only B >= A (type I)
// or B > A (type II).  This visits exactly the (cell pair, bucket pair) items
// of the recursion, in a different order.  Neighbour and parent-neighbour cells
// are formed by dilated (per-dimension masked) addition on Morton codes.
//
// Decisions are made in single precision with a rigorous error band; inside
// the band they are recomputed with the exact FP64 rule (the same arithmetic
// as the FP64 reference), so the edge set equals the FP64 one.  The kernels are
// instantiated per dimension (d = 1..4, and a generic d <= 8).
#include "internal.cuh"
#include "kernels.h"

namespace gg {

// ------------------------------------------------------------------ per-pair decisions
// Per-thread event counts (statistics), summed per warp at the end of a kernel.
struct Counters {
    uint32_t t1pairs = 0, coins = 0, recheck = 0, t2items = 0, draws = 0, cands = 0;
};

struct View {  // per-vertex arrays indexed by position
    const uint32_t* X;
    const float* sv;
    const double* w;      // GIRG weights or HRG radii
    const uint32_t* ids;  // nullptr: id = position
    const float* E32;
    const float* einv32;
    const float* sh32;
    int64_t n;
    const uint4* rec;     // packed GIRG records (d <= 4), or nullptr: the arrays above
    const uint4* hrec;    // packed HRG records, or nullptr: X, E32, einv32, sh32
};

__device__ __forceinline__ View sorted_view(const DevCfg& cfg) {
    return View{cfg.Xs, cfg.sv, cfg.ws, cfg.ids, cfg.E32, cfg.einv32, cfg.sh32, cfg.n, cfg.vrec, cfg.hrec};
}

// What a single-precision HRG decision reads of one vertex: its angle, e^r, e^-r and
// sinh r, from one 16-byte record when the view has them.
struct HRec {
    uint32_t X;
    float E, ei, sh;
};

__device__ __forceinline__ HRec load_hrec(const View& V, uint32_t p) {
    if (V.hrec) {
        const uint4 a = __ldg(V.hrec + p);
        return HRec{a.x, __uint_as_float(a.y), __uint_as_float(a.z), __uint_as_float(a.w)};
    }
    return HRec{V.X[p], V.E32[p], V.einv32[p], V.sh32[p]};
}

__device__ __forceinline__ uint32_t vid(const View& V, uint32_t p) { return V.ids ? V.ids[p] : p; }

// What a GIRG decision reads of one vertex: its coordinates, its single-precision scale
// and its original id.  From a packed record (one 16-byte load for d <= 2, two for
// d = 3, 4) when the view has them, else from the separate arrays.
template <int DIM>
struct VRec {
    uint32_t x[DIM];
    float s;
    uint32_t id;
};

template <int DIM>
__device__ __forceinline__ VRec<DIM> load_rec(const View& V, uint32_t p) {
    static_assert(DIM >= 1 && DIM <= 4, "packed records hold up to four coordinates");
    VRec<DIM> r;
    if (V.rec) {
        if constexpr (DIM <= 2) {
            const uint4 a = __ldg(V.rec + p);
            r.x[0] = a.x;
            if constexpr (DIM == 2) r.x[1] = a.y;
            r.s = __uint_as_float(a.z);
            r.id = a.w;
        } else {
            const uint4 a = __ldg(V.rec + 2 * (size_t)p), b = __ldg(V.rec + 2 * (size_t)p + 1);
            r.x[0] = a.x;
            r.x[1] = a.y;
            r.x[2] = a.z;
            if constexpr (DIM == 4) r.x[3] = a.w;
            r.s = __uint_as_float(b.x);
            r.id = b.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DIM; ++k) r.x[k] = V.X[(int64_t)k * V.n + p];
        r.s = V.sv[p];
        r.id = vid(V, p);
    }
    return r;
}

template <int DIM>
__device__ __forceinline__ uint32_t rec_D(const VRec<DIM>& a, const VRec<DIM>& b) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const uint32_t t = circ_diff(a.x[k], b.x[k]);
        m = t > m ? t : m;
    }
    return m;
}

template <int DIM>
__device__ __forceinline__ uint32_t torus_D(int d, const View& V, uint32_t pu, uint32_t pv) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < (DIM ? DIM : kMaxDim); ++k) {
        if (DIM == 0 && k >= d) break;
        const uint32_t t = circ_diff(V.X[(int64_t)k * V.n + pu], V.X[(int64_t)k * V.n + pv]);
        m = t > m ? t : m;
    }
    return m;
}

// kappa_uv / r in single precision (D > 0).
__device__ __forceinline__ float kappa_ratio(const View& V, uint32_t pu, uint32_t pv, uint32_t D) {
    return V.sv[pu] * V.sv[pv] * __fdividef(4294967296.0f, __uint2float_rn(D));
}

__device__ __forceinline__ double girg_p_pair(const DevCfg& cfg, const View& V, uint32_t pu,
                                              uint32_t pv, uint32_t D) {
    return girg_p64(V.w[pu], V.w[pv], D, cfg.W, cfg.K, cfg.invT, cfg.m_int, cfg.d);
}

// HRG cosh d in FP64 from the radii of both vertices.
__device__ __noinline__ double hrg_coshd_pair(const View& V, uint32_t pu, uint32_t pv, uint32_t D) {
    double Eu, shu, Ev, shv;
    hrg_vertex64(V.w[pu], &Eu, &shu);
    hrg_vertex64(V.w[pv], &Ev, &shv);
    return hrg_coshd64(Eu, shu, Ev, shv, D);
}

__device__ __noinline__ bool girg_t1_exact(const DevCfg& cfg, const View& V, uint32_t pu,
                                           uint32_t pv, uint32_t D, uint32_t lo, uint32_t hi) {
    if (cfg.tzero) return girg_thresh64(V.w[pu], V.w[pv], D, cfg.W, cfg.K, cfg.d);
    return uniform53(lo, hi) < girg_p_pair(cfg, V, pu, pv, D);
}

__device__ __noinline__ bool hrg_t1_exact(const DevCfg& cfg, const View& V, uint32_t pu, uint32_t pv,
                                          uint32_t D, uint32_t lo, uint32_t hi) {
    const double cd = hrg_coshd_pair(V, pu, pv, D);
    if (cfg.tzero) return cd < cfg.coshR;
    return uniform53(lo, hi) < hrg_p_from_coshd(cd, cfg.R, cfg.T);
}

__device__ __noinline__ bool t2_exact(const DevCfg& cfg, const View& V, uint32_t pu, uint32_t pv,
                                      uint32_t D, uint32_t lo, uint32_t hi, double pbar) {
    double p;
    if (cfg.model == 0)
        p = D == 0 ? 1.0 : girg_p_pair(cfg, V, pu, pv, D);
    else
        p = hrg_p_from_coshd(hrg_coshd_pair(V, pu, pv, D), cfg.R, cfg.T);
    return DMUL(uniform53(lo, hi), pbar) < p;
}

// cosh d of two HRG vertices in single precision from their records (D: angle gap).
__device__ __forceinline__ float hrg_coshd32_rec(const HRec& u, const HRec& v, uint32_t D) {
    const float s = sinpif(__uint2float_rn(D) * 0x1p-32f);
    const float ch = 0.5f * (u.E * v.ei + v.E * u.ei);
    return ch + 2.0f * u.sh * v.sh * (s * s);
}

__device__ __forceinline__ float hrg_coshd32(const View& V, uint32_t pu, uint32_t pv, uint32_t D) {
    return hrg_coshd32_rec(load_hrec(V, pu), load_hrec(V, pv), D);
}

__device__ __forceinline__ float hrg_p32(const DevCfg& cfg, float cd) {
    return 1.0f / (expf((acoshf(cd) - cfg.R32) * cfg.inv2T32) + 1.0f);
}

// Type I: edge iff U(seed, u, v) < p_uv (T > 0) or the threshold rule (T = 0).  The
// pair's original ids go to *ida, *idb (ida < idb).
template <int DIM>
__device__ bool decide_t1(const DevCfg& cfg, const View& V, uint32_t pu, uint32_t pv, Counters& C,
                          uint32_t* ida, uint32_t* idb) {
    if constexpr (DIM >= 1 && DIM <= 4) {
        if (cfg.model == 0) {  // GIRG from the two vertex records
            const VRec<DIM> ru = load_rec<DIM>(V, pu), rv = load_rec<DIM>(V, pv);
            const uint32_t a = ru.id < rv.id ? ru.id : rv.id, b = ru.id < rv.id ? rv.id : ru.id;
            *ida = a;
            *idb = b;
            const uint32_t D = rec_D<DIM>(ru, rv);
            if (D == 0) return true;
            if (cfg.precision == 1) {
                uint32_t lo = 0, hi = 0;
                if (!cfg.tzero) {
                    ++C.coins;
                    const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
                    lo = o.x;
                    hi = o.y;
                }
                return girg_t1_exact(cfg, V, pu, pv, D, lo, hi);
            }
            const float ratio = ru.s * rv.s * __fdividef(4294967296.0f, __uint2float_rn(D));
            if (cfg.tzero) {
                if (ratio > 1.0f + cfg.band_ratio) return true;
                if (ratio < 1.0f - cfg.band_ratio) return false;
                ++C.recheck;
                return girg_t1_exact(cfg, V, pu, pv, D, 0u, 0u);
            }
            if (ratio >= 1.0f + cfg.band_ratio) return true;  // p = 1
            const float lp = cfg.dT * __log2f(ratio);        // log2 p
            if (lp < -54.0f - cfg.bandG) return false;        // p < 2^-54 < every U
            ++C.coins;
            const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
            const float G = lp - log2_uniform32(o.x, o.y);
            if (G > cfg.bandG) return true;
            if (G < -cfg.bandG) return false;
            ++C.recheck;
            return girg_t1_exact(cfg, V, pu, pv, D, o.x, o.y);
        }
    }
    const uint32_t iu = vid(V, pu), iv = vid(V, pv);
    const uint32_t a = iu < iv ? iu : iv, b = iu < iv ? iv : iu;
    *ida = a;
    *idb = b;
    if ((DIM == 1 || DIM == 0) && cfg.model == 1) {
        // HRG (Sec. 2.2): threshold d < R, binomial U < p_T(d)
        const uint32_t D = circ_diff(V.X[pu], V.X[pv]);
        if (cfg.precision == 1) {
            uint32_t lo = 0, hi = 0;
            if (!cfg.tzero) {
                ++C.coins;
                const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
                lo = o.x;
                hi = o.y;
            }
            return hrg_t1_exact(cfg, V, pu, pv, D, lo, hi);
        }
        const float cd = hrg_coshd32(V, pu, pv, D);
        if (cfg.tzero) {
            if (cd < cfg.coshR32 * (1.0f - 0x1p-16f)) return true;
            if (cd > cfg.coshR32 * (1.0f + 0x1p-16f)) return false;
            ++C.recheck;
            return hrg_t1_exact(cfg, V, pu, pv, D, 0u, 0u);
        }
        ++C.coins;
        const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
        // distance filter (Sec. 4.3): the bin of U brackets the threshold on cosh d;
        // bin m = floor(U (K - 1)) exactly, from the 53-bit integer of U
        const unsigned long long odd = 2ull * ((((unsigned long long)o.y << 32) | o.x) >> 12) + 1ull;
        const int m = (int)((odd * (unsigned long long)(cfg.filt_k - 1)) >> 53);
        if (cd * (1.0f + 0x1p-16f) < cfg.filt_lo[m + 1]) return true;
        if (cd * (1.0f - 0x1p-16f) >= cfg.filt_hi[m]) return false;
        const float p32 = hrg_p32(cfg, cd);
        const float u32 = uniform32(o.x, o.y);
        if (u32 < p32 * (1.0f - cfg.bandG)) return true;
        if (u32 > p32 * (1.0f + cfg.bandG)) return false;
        ++C.recheck;
        return hrg_t1_exact(cfg, V, pu, pv, D, o.x, o.y);
    }
    const uint32_t D = torus_D<DIM>(cfg.d, V, pu, pv);
    if (D == 0) return true;
    if (cfg.precision == 1) {
        uint32_t lo = 0, hi = 0;
        if (!cfg.tzero) {
            ++C.coins;
            const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
            lo = o.x;
            hi = o.y;
        }
        return girg_t1_exact(cfg, V, pu, pv, D, lo, hi);
    }
    const float ratio = kappa_ratio(V, pu, pv, D);
    if (cfg.tzero) {
        if (ratio > 1.0f + cfg.band_ratio) return true;
        if (ratio < 1.0f - cfg.band_ratio) return false;
        ++C.recheck;
        return girg_t1_exact(cfg, V, pu, pv, D, 0u, 0u);
    }
    if (ratio >= 1.0f + cfg.band_ratio) return true;  // p = 1
    const float lp = cfg.dT * __log2f(ratio);        // log2 p (ratio < 2^-126 gives -inf)
    if (lp < -54.0f - cfg.bandG) return false;        // p < 2^-54 < every U
    ++C.coins;
    const P4 o = philox(a, b, kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
    const float G = lp - log2_uniform32(o.x, o.y);
    if (G > cfg.bandG) return true;
    if (G < -cfg.bandG) return false;
    ++C.recheck;
    return girg_t1_exact(cfg, V, pu, pv, D, o.x, o.y);
}

// NP type-I pairs per lane (GIRG, packed records, single-precision decisions): their
// vertex records load together and the coins' Philox rounds are independent, so a lane
// carries NP dependency chains.  The decisions are those of decide_t1; a
// coin is computed for every pair (about 93% need one) but counted only when used.
template <int DIM, int NP>
__device__ __forceinline__ void decide_t1_xp(const DevCfg& cfg, const View& V, const bool (&ok)[NP],
                                             const uint32_t (&pu)[NP], const uint32_t (&pv)[NP],
                                             Counters& C, bool (&edge)[NP], uint32_t (&ida)[NP],
                                             uint32_t (&idb)[NP]) {
    VRec<DIM> ru[NP], rv[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        ru[h] = load_rec<DIM>(V, ok[h] ? pu[h] : 0u);
        rv[h] = load_rec<DIM>(V, ok[h] ? pv[h] : 0u);
    }
    uint32_t D[NP];
    P4 o[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        ida[h] = ru[h].id < rv[h].id ? ru[h].id : rv[h].id;
        idb[h] = ru[h].id < rv[h].id ? rv[h].id : ru[h].id;
        D[h] = rec_D<DIM>(ru[h], rv[h]);
    }
    if (!cfg.tzero) {
#pragma unroll
        for (int h = 0; h < NP; ++h) o[h] = philox(ida[h], idb[h], kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
    }
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        edge[h] = false;
        if (!ok[h]) continue;
        if (D[h] == 0) {
            edge[h] = true;
            continue;
        }
        const float ratio = ru[h].s * rv[h].s * __fdividef(4294967296.0f, __uint2float_rn(D[h]));
        if (cfg.tzero) {
            if (ratio > 1.0f + cfg.band_ratio) {
                edge[h] = true;
            } else if (!(ratio < 1.0f - cfg.band_ratio)) {
                ++C.recheck;
                edge[h] = girg_t1_exact(cfg, V, pu[h], pv[h], D[h], 0u, 0u);
            }
            continue;
        }
        if (ratio >= 1.0f + cfg.band_ratio) {  // p = 1
            edge[h] = true;
            continue;
        }
        const float lp = cfg.dT * __log2f(ratio);  // log2 p
        if (lp < -54.0f - cfg.bandG) continue;     // p < 2^-54 < every U
        ++C.coins;
        const float G = lp - log2_uniform32(o[h].x, o[h].y);
        if (G > cfg.bandG) {
            edge[h] = true;
        } else if (!(G < -cfg.bandG)) {
            ++C.recheck;
            edge[h] = girg_t1_exact(cfg, V, pu[h], pv[h], D[h], o[h].x, o[h].y);
        }
    }
}

// The same for HRG pairs (single-precision decisions): the angles, radial terms and ids
// of all NP pairs load together and their coins' Philox rounds interleave; the
// decisions are those of decide_t1.
template <int NP>
__device__ __forceinline__ void decide_t1_hrg_xp(const DevCfg& cfg, const View& V,
                                                 const bool (&ok)[NP], const uint32_t (&pu)[NP],
                                                 const uint32_t (&pv)[NP], Counters& C,
                                                 bool (&edge)[NP], uint32_t (&ida)[NP],
                                                 uint32_t (&idb)[NP]) {
    uint32_t D[NP];
    float cd[NP];
    P4 o[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        const uint32_t u = ok[h] ? pu[h] : 0u, v = ok[h] ? pv[h] : 0u;
        const uint32_t iu = vid(V, u), iv = vid(V, v);
        ida[h] = iu < iv ? iu : iv;
        idb[h] = iu < iv ? iv : iu;
        const HRec ru = load_hrec(V, u), rv = load_hrec(V, v);
        D[h] = circ_diff(ru.X, rv.X);
        cd[h] = hrg_coshd32_rec(ru, rv, D[h]);
    }
    if (!cfg.tzero) {
#pragma unroll
        for (int h = 0; h < NP; ++h) o[h] = philox(ida[h], idb[h], kTagPair, 0u, cfg.seed_lo, cfg.seed_hi);
    }
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        edge[h] = false;
        if (!ok[h]) continue;
        if (cfg.tzero) {
            if (cd[h] < cfg.coshR32 * (1.0f - 0x1p-16f)) {
                edge[h] = true;
            } else if (!(cd[h] > cfg.coshR32 * (1.0f + 0x1p-16f))) {
                ++C.recheck;
                edge[h] = hrg_t1_exact(cfg, V, pu[h], pv[h], D[h], 0u, 0u);
            }
            continue;
        }
        ++C.coins;
        // distance filter (Sec. 4.3): the bin of U brackets the threshold on cosh d;
        // bin m = floor(U (K - 1)) exactly, from the 53-bit integer of U
        const unsigned long long odd =
            2ull * ((((unsigned long long)o[h].y << 32) | o[h].x) >> 12) + 1ull;
        const int m = (int)((odd * (unsigned long long)(cfg.filt_k - 1)) >> 53);
        if (cd[h] * (1.0f + 0x1p-16f) < cfg.filt_lo[m + 1]) {
            edge[h] = true;
            continue;
        }
        if (cd[h] * (1.0f - 0x1p-16f) >= cfg.filt_hi[m]) continue;
        const float p32 = hrg_p32(cfg, cd[h]);
        const float u32 = uniform32(o[h].x, o[h].y);
        if (u32 < p32 * (1.0f - cfg.bandG)) {
            edge[h] = true;
        } else if (!(u32 > p32 * (1.0f + cfg.bandG))) {
            ++C.recheck;
            edge[h] = hrg_t1_exact(cfg, V, pu[h], pv[h], D[h], o[h].x, o[h].y);
        }
    }
}

// Type-II acceptance: accept iff U' pbar < p_uv.
template <int DIM>
__device__ bool accept_t2(const DevCfg& cfg, const View& V, uint32_t pu, uint32_t pv, uint32_t lo,
                          uint32_t hi, const TwoEntry& e, Counters& C) {
    if ((DIM == 1 || DIM == 0) && cfg.model == 1) {
        const HRec ru = load_hrec(V, pu), rv = load_hrec(V, pv);
        const uint32_t D = circ_diff(ru.X, rv.X);
        if (cfg.precision == 1) return t2_exact(cfg, V, pu, pv, D, lo, hi, e.pbar);
        const float p32 = hrg_p32(cfg, hrg_coshd32_rec(ru, rv, D));
        const float up = uniform32(lo, hi) * exp2f(e.log2pbar);
        if (up < p32 * (1.0f - cfg.bandG)) return true;
        if (up > p32 * (1.0f + cfg.bandG)) return false;
        ++C.recheck;
        return t2_exact(cfg, V, pu, pv, D, lo, hi, e.pbar);
    }
    const uint32_t D = torus_D<DIM>(cfg.d, V, pu, pv);
    if (cfg.precision == 1) return t2_exact(cfg, V, pu, pv, D, lo, hi, e.pbar);
    if (D == 0) return true;
    const float ratio = kappa_ratio(V, pu, pv, D);
    if (ratio >= 1.0f + cfg.band_ratio) return true;
    if (ratio < 0x1p-126f) {  // subnormal: no relative error bound in single precision
        ++C.recheck;
        return t2_exact(cfg, V, pu, pv, D, lo, hi, e.pbar);
    }
    const float G = cfg.dT * __log2f(ratio) - log2_uniform32(lo, hi) - e.log2pbar;
    if (G > cfg.bandG) return true;
    if (G < -cfg.bandG) return false;
    ++C.recheck;
    return t2_exact(cfg, V, pu, pv, D, lo, hi, e.pbar);
}


// The fast-path fields of a TwoEntry a type-II lane keeps; the FP64 fields are
// reloaded from the table in the rare fallback paths.
struct TwoFast {
    float invLb, log2pbar;
    uint32_t tii;
    bool one;
};

// The geometric jump of one draw (Sec. 3.2): 0 stop, 1 continue with *X.
__device__ __forceinline__ int draw_jump_fast(const DevCfg& cfg, const TwoFast& e, const P4& o,
                                              unsigned long long rem, unsigned long long* X,
                                              Counters& C) {
    *X = 0;
    if (e.one) return rem == 0 ? 0 : 1;
    int r = 2;
    if (cfg.precision == 0) r = jump32(o.x, o.y, e.invLb, rem, X);
    if (r == 2) {
        if (cfg.precision == 0) ++C.recheck;
        r = jump64(o.x, o.y, cfg.tii[e.tii].Lb, rem, X);
    }
    return r;
}

template <int DIM, bool HRG = false>
__device__ __forceinline__ bool accept_t2_fast(const DevCfg& cfg, const View& V, uint32_t pu,
                                               uint32_t pv, uint32_t lo, uint32_t hi,
                                               const TwoFast& e, Counters& C, uint32_t* idu,
                                               uint32_t* idv) {
    if constexpr (HRG) {  // the HRG instantiation (d = 1)
        *idu = vid(V, pu);
        *idv = vid(V, pv);
        return accept_t2<DIM>(cfg, V, pu, pv, lo, hi, cfg.tii[e.tii], C);
    }
    if constexpr (DIM >= 1 && DIM <= 4) {
        if (cfg.model == 0) {  // GIRG from the two vertex records
            const VRec<DIM> ru = load_rec<DIM>(V, pu), rv = load_rec<DIM>(V, pv);
            *idu = ru.id;
            *idv = rv.id;
            const uint32_t D = rec_D<DIM>(ru, rv);
            if (cfg.precision == 1) return t2_exact(cfg, V, pu, pv, D, lo, hi, cfg.tii[e.tii].pbar);
            if (D == 0) return true;
            const float ratio = ru.s * rv.s * __fdividef(4294967296.0f, __uint2float_rn(D));
            if (ratio >= 1.0f + cfg.band_ratio) return true;
            if (ratio >= 0x1p-126f) {
                const float G = cfg.dT * __log2f(ratio) - log2_uniform32(lo, hi) - e.log2pbar;
                if (G > cfg.bandG) return true;
                if (G < -cfg.bandG) return false;
            }  // else subnormal: no relative error bound in single precision
            ++C.recheck;
            return t2_exact(cfg, V, pu, pv, D, lo, hi, cfg.tii[e.tii].pbar);
        }
    }
    *idu = vid(V, pu);
    *idv = vid(V, pv);
    const uint32_t D = torus_D<DIM>(cfg.d, V, pu, pv);
    if (cfg.precision == 1) return t2_exact(cfg, V, pu, pv, D, lo, hi, cfg.tii[e.tii].pbar);
    if (D == 0) return true;
    const float ratio = kappa_ratio(V, pu, pv, D);
    if (ratio >= 1.0f + cfg.band_ratio) return true;
    if (ratio >= 0x1p-126f) {
        const float G = cfg.dT * __log2f(ratio) - log2_uniform32(lo, hi) - e.log2pbar;
        if (G > cfg.bandG) return true;
        if (G < -cfg.bandG) return false;
    }  // else subnormal: no relative error bound in single precision
    ++C.recheck;
    return t2_exact(cfg, V, pu, pv, D, lo, hi, cfg.tii[e.tii].pbar);
}

__device__ __forceinline__ void flush_counters(const DevCfg& cfg, const Counters& C) {
    unsigned long long v[6] = {C.t1pairs, C.coins, C.recheck, C.t2items, C.draws, C.cands};
    const int idx[6] = {kStatT1Pairs, kStatCoins, kStatRecheck, kStatT2Items, kStatDraws, kStatCands};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        unsigned long long x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&cfg.stats[idx[q]], x);
    }
}

// ------------------------------------------------------------------ rows
// Row heads: the first sorted position of every non-empty (bucket i, level l, cell)
// for l <= CLd(i) (the deepest comparison level of i with a bucket j >= i).  Each
// row becomes one work entry per bucket it pairs with: type-II entries (distant
// cells) and type-I entries (neighbour cells) in separate lists; an entry packs
// p | l << 32 | i << 38 | e << 44 (e: index of the bucket in the row's class).
__device__ __forceinline__ uint64_t pack_entry(uint32_t p, int l, int i, uint32_t e) {
    return (uint64_t)p | ((uint64_t)l << 32) | ((uint64_t)i << 38) | ((uint64_t)e << 44);
}

// Block-wide slot allocation: each thread passes its counts x[q]; one atomicAdd per
// counter and block (a same-address atomic per warp serialises in L2 and dominated
// the enumeration kernels).  Returns each thread's first slot per counter.  Every
// thread of a block of kAllocThreads must call it.
constexpr int kAllocThreads = 256;

template <int NQ, class C>
__device__ __forceinline__ void block_alloc(const uint32_t (&x)[NQ], C* const (&ctr)[NQ],
                                            C (&base)[NQ]) {
    constexpr int NW = kAllocThreads / 32;
    __shared__ C s_w[NW][NQ];
    __shared__ C s_b[NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        incl[q] = x[q];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl[q], o);
            if (lane >= o) incl[q] += t;
        }
        if (lane == 31) s_w[warp][q] = (C)incl[q];
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        C acc = 0;
        for (int w = 0; w < NW; ++w) {
            const C t = s_w[w][q];
            s_w[w][q] = acc;
            acc += t;
        }
        s_b[q] = acc ? atomicAdd(ctr[q], acc) : (C)0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; ++q) base[q] = s_b[q] + s_w[warp][q] + (C)(incl[q] - x[q]);
    __syncthreads();  // s_w and s_b are reused by the next call
}

__global__ void __launch_bounds__(kAllocThreads) k_rows(DevCfg cfg) {
    const int64_t n = cfg.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x; p0 < n; p0 += stride) {
        const int64_t p = p0 + threadIdx.x;
        int i = 0, top = -1;
        uint32_t cell = 0, prev = 0;
        bool first = false;
        if (p < n) {
            i = cfg.slayer[p];
            const uint32_t base = cfg.layer_base[i];
            cell = cfg.skey[p] - base;
            first = (uint32_t)p == cfg.lstart[i];
            prev = first ? 0u : cfg.skey[p - 1] - base;
            top = cfg.CLd[i];
        }
        // p heads its cell on level l iff the cells of p - 1 and p differ there, i.e. for
        // every l >= l0 with l0 from the highest differing bit of the two keys (a key of
        // bucket i has d I(i) bits, level l keeps the top d l of them)
        int l0 = top + 1;
        if (p < n) {
            const uint32_t diff = cell ^ prev;
            if (first)
                l0 = 0;
            else if (diff)
                l0 = cfg.I[i] - (31 - __clz(diff)) / cfg.d;
            if (l0 < 0) l0 = 0;
        }
        uint32_t heads = 0, m2 = 0, m1 = 0;
        for (int l = l0; l <= top; ++l) {
            const RowClass rc = cfg.classes[(uint32_t)i * (kMaxLevel + 1) + l];
            ++heads;
            m2 += rc.n2;
            m1 += rc.n1;
        }
        const uint32_t cnt[3] = {heads, m2, m1};
        unsigned int* const ctr[3] = {cfg.row_count, cfg.ent2_count, cfg.ent1_count};
        unsigned int slot[3];
        block_alloc<3>(cnt, ctr, slot);
        uint32_t b2 = slot[1], b1 = slot[2];
        for (int l = l0; l <= top; ++l) {
            const RowClass rc = cfg.classes[(uint32_t)i * (kMaxLevel + 1) + l];
            for (uint32_t e = 0; e < rc.n2; ++e, ++b2)
                if (b2 < cfg.ent2_cap) cfg.ent2[b2] = pack_entry((uint32_t)p, l, i, e);
            for (uint32_t e = 0; e < rc.n1; ++e, ++b1)
                if (b1 < cfg.ent1_cap) cfg.ent1[b1] = pack_entry((uint32_t)p, l, i, e);
        }
    }
}

// ------------------------------------------------------------------ enumeration
constexpr int kEnumThreads = 256;
static_assert(kEnumThreads == kAllocThreads, "the enumeration allocates slots per block");
constexpr int kWarps = kEnumThreads / 32;
constexpr uint32_t kSplitB = 1024, kSplitAB = 4096;

// floor(a / b) for a < 2^24 and b >= 1 with a / b < 2^23: a float reciprocal estimate
// (within one of the quotient there), corrected by one step.
__device__ __forceinline__ uint32_t udiv24(uint32_t a, uint32_t b) {
    uint32_t q = __float2uint_rz(__uint2float_rn(a) * __frcp_rn(__uint2float_rn(b)));
    const int r = (int)a - (int)(q * b);
    if (r < 0)
        --q;
    else if (r >= (int)b)
        ++q;
    return q;
}

// An offset digit e in {-1, 0, 1} is a distinct neighbour on a level with 2^lev cells
// per dimension unless the grid is too small: 1 cell -> only 0; 2 cells -> not -1.
__device__ __forceinline__ bool digit_ok(int e, int lev) {
    if (lev == 0) return e == 0;
    if (lev == 1) return e != -1;
    return true;
}

// Add e in {-1, 0, 1} to the coordinate held in the Morton bits `mask` of M (one
// dimension); carries run through the other dimensions' bits, so the result wraps
// on the torus.
__device__ __forceinline__ uint32_t dil_add(uint32_t M, uint32_t mask, uint32_t unit, int e) {
    const uint32_t x = M & mask;
    if (e > 0) return ((x | ~mask) + unit) & mask;
    if (e < 0) return (x - unit) & mask;
    return x;
}

// Bits of dimension k (coordinate 0 most significant) of a Morton code at level l.
__device__ __forceinline__ uint32_t dim_mask(int d, int k, int l) {
    const int nb = d * l;  // <= 32
    const uint32_t lowk = 1u << (d - 1 - k);
    uint32_t pat;  // bits d-1-k, 2d-1-k, ... of a 32-bit word
    switch (d) {
        case 1: pat = 0xffffffffu; break;
        case 2: pat = 0x55555555u << (1 - k); break;
        case 3: pat = 0x49249249u << (2 - k); break;
        case 4: pat = 0x11111111u << (3 - k); break;
        default: {
            pat = 0;
            for (int b = 0; b * d < 32; ++b) pat |= lowk << (b * d);
        }
    }
    return nb >= 32 ? pat : (pat & ((1u << nb) - 1u));
}

// The cell, range and geometry of a work entry.
struct EntryCtx {
    uint32_t A, a_lo, a_len;
    int l, i, j;
    uint32_t e;
    RowClass rc;
    uint32_t baseB;  // global cell index base of bucket j
    int sB;          // shift from level l to bucket j's insertion level
};

template <int DIM>
__device__ __forceinline__ EntryCtx decode_entry(const DevCfg& cfg, uint64_t ent, int d, bool type1) {
    EntryCtx x;
    const uint32_t p = (uint32_t)ent;
    x.l = (int)((ent >> 32) & 0x3f);
    x.i = (int)((ent >> 38) & 0x3f);
    x.e = (uint32_t)(ent >> 44);
    x.rc = cfg.classes[(uint32_t)x.i * (kMaxLevel + 1) + x.l];
    x.j = cfg.jlist[x.rc.jbase + (type1 ? x.rc.n2 : 0u) + x.e];
    const uint32_t base_i = cfg.layer_base[x.i];
    const int sA = d * (cfg.I[x.i] - x.l);
    x.A = (uint32_t)((uint64_t)(cfg.skey[p] - base_i) >> sA);
    x.a_lo = cfg.offs[base_i + (uint32_t)((uint64_t)x.A << sA)];
    x.a_len = cfg.offs[base_i + (uint32_t)(((uint64_t)x.A + 1) << sA)] - x.a_lo;
    x.baseB = cfg.layer_base[x.j];
    x.sB = d * (cfg.I[x.j] - x.l);
    return x;
}

__device__ __forceinline__ void range_of(const DevCfg& cfg, const EntryCtx& x, uint32_t B,
                                         uint32_t* lo, uint32_t* len) {
    const uint32_t a = cfg.offs[x.baseB + (uint32_t)((uint64_t)B << x.sB)];
    *lo = a;
    *len = cfg.offs[x.baseB + (uint32_t)(((uint64_t)B + 1) << x.sB)] - a;
}

// Distances in cells along one dimension between A and the children of its parent's
// neighbours: 3 bits for child position 2 (e + 1) + kid, where e in {-1, 0, 1} is the
// parent offset and kid the child bit; A's own child bit alpha fixes the row
// (alpha 0: 2 1 0 1 2 3, alpha 1: 3 2 1 0 1 2).  With 4 cells per dimension (level 2)
// a distance of 3 wraps around the torus to 1.
__host__ __device__ constexpr uint32_t pack6(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                             uint32_t e, uint32_t f) {
    return a | b << 3 | c << 6 | d << 9 | e << 12 | f << 15;
}
__device__ __forceinline__ uint32_t child_dists(uint32_t alpha, bool four) {
    if (alpha) return four ? pack6(1, 2, 1, 0, 1, 2) : pack6(3, 2, 1, 0, 1, 2);
    return four ? pack6(2, 1, 0, 1, 2, 1) : pack6(2, 1, 0, 1, 2, 3);
}

// The children (d-bit numbers, dimension 0 most significant) whose bit of dimension k
// is set, as a bit set over the 2^d children (d <= 5).
__device__ __forceinline__ uint32_t kids_with_bit(int d, int k) {
    const int b = d - 1 - k;
    const uint32_t pat = b == 0 ? 0xAAAAAAAAu : b == 1 ? 0xCCCCCCCCu : b == 2 ? 0xF0F0F0F0u
                       : b == 3 ? 0xFF00FF00u : 0xFFFF0000u;
    return d >= 5 ? pat : pat & ((1u << (1u << d)) - 1u);
}

// Visit the distant partner cells B of A (children of the neighbours of A's
// parent, not neighbours of A) that count for bucket j and hold a vertex of it:
// f(B, g, lo, len, rank) with the gap g = L_inf distance - 1 in {1, 2}, the range of
// sorted positions (len > 0) and the rank, in rank order, rank = (sum_k (e_k + 1)
// 3^(d-1-k)) 2^d + sum_k kid_k 2^(d-1-k).  The 2^d children of a parent neighbour are consecutive
// cells with 2^d + 1 consecutive offsets.  The parent neighbours go in groups of
// three that differ in the last digit only: the first and end offsets of a group are
// loaded together, then (d <= 3) the inner offsets of its non-empty members, so a
// group costs two dependent loads.  For d <= 4 the distant children of a parent
// neighbour and their gaps come from per-dimension bit sets of the children.
template <int DIM, class F>
__device__ __forceinline__ void for_partners(const DevCfg& cfg, const EntryCtx& x, int d, F f) {
    constexpr int DM = DIM ? DIM : kMaxDim;
    constexpr uint32_t NG = DIM == 1 ? 1u : DIM == 2 ? 3u : DIM == 3 ? 9u : DIM == 4 ? 27u : 0u;
    constexpr bool kMasks = DIM >= 1 && DIM <= 4;  // 2^d <= 16 children per bit set
    constexpr bool kBatch = DIM >= 1 && DIM <= 3;  // inner offsets of a group in registers
    constexpr int NKB = DIM >= 1 && DIM <= 3 ? (1 << DIM) - 1 : 1;
    uint32_t ng = NG;
    if (DIM == 0) {
        ng = 1;
        for (int k = 1; k < d; ++k) ng *= 3u;
    }
    const uint32_t nk = 1u << d;
    const uint32_t PA = x.A >> d;
    const int lev = x.l - 1;  // the parents' level: 1 cell (only e = 0) or 2 (no e = -1)
    const bool four = x.l == 2;
    const bool same = x.j == x.i;  // only B > A
    uint32_t pm[DM], p0[DM], pp[DM], dist[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
        if (k >= d) break;
        const uint32_t mask = dim_mask(d, k, lev), unit = 1u << (d - 1 - k);
        pm[k] = dil_add(PA, mask, unit, -1);
        p0[k] = PA & mask;
        pp[k] = dil_add(PA, mask, unit, 1);
        dist[k] = child_dists((x.A >> (d - 1 - k)) & 1u, four);
    }
    auto offs_at = [&](uint32_t cell) {
        return cfg.offs[x.baseB + (uint32_t)((uint64_t)cell << x.sB)];
    };
    const int kl = d - 1;  // the dimension whose digit varies within a group
#pragma unroll(DIM == 1 || DIM == 2 ? NG : 1)
    for (uint32_t gi = 0; gi < ng; ++gi) {
        int ek[DM];
        uint32_t q = gi, Pg = 0;
        bool okg = true, anyg = false;
#pragma unroll
        for (int k = DM - 1; k >= 0; --k) {
            ek[k] = 0;
            if (k >= kl) continue;
            ek[k] = (int)(q % 3u) - 1;
            q /= 3u;
            okg = okg && digit_ok(ek[k], lev);
            anyg = anyg || ek[k] != 0;  // the own parent has only neighbour children
            Pg |= ek[k] < 0 ? pm[k] : ek[k] > 0 ? pp[k] : p0[k];
        }
        if (!okg) continue;
        uint32_t first[3], lo0[3], end[3];
        bool use[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int e = t - 1;
            first[t] = (Pg | (e < 0 ? pm[kl] : e > 0 ? pp[kl] : p0[kl])) << d;
            use[t] = digit_ok(e, lev) && (anyg || e != 0) && !(same && first[t] < x.A);
            lo0[t] = 0;
            end[t] = 0;
            if (use[t]) {
                lo0[t] = offs_at(first[t]);
                end[t] = offs_at(first[t] + nk);
            }
        }
        uint32_t mid[3][NKB];
        if constexpr (kBatch) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (use[t] && lo0[t] != end[t]) {
#pragma unroll
                    for (int c = 0; c < NKB; ++c) mid[t][c] = offs_at(first[t] + (uint32_t)c + 1u);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (!use[t] || lo0[t] == end[t]) continue;  // no vertex of bucket j here
            ek[kl] = t - 1;
            if constexpr (kMasks) {
                uint32_t far = 0, far3 = 0;  // children at distance >= 2 (>= 3) in some dimension
#pragma unroll
                for (int k = 0; k < DM; ++k) {
                    const uint32_t s = 6u * (uint32_t)(ek[k] + 1);
                    const uint32_t d0 = (dist[k] >> s) & 7u, d1 = (dist[k] >> (s + 3u)) & 7u;
                    const uint32_t m1 = kids_with_bit(d, k), m0 = ~m1 & ((1u << nk) - 1u);
                    far |= (d0 >= 2u ? m0 : 0u) | (d1 >= 2u ? m1 : 0u);
                    far3 |= (d0 >= 3u ? m0 : 0u) | (d1 >= 3u ? m1 : 0u);
                }
                uint32_t lo = lo0[t];
#pragma unroll
                for (uint32_t kid = 0; kid < (1u << DM); ++kid) {
                    uint32_t hi;
                    if constexpr (kBatch)
                        hi = kid + 1 < nk ? mid[t][kid < (uint32_t)NKB ? kid : 0] : end[t];
                    else
                        hi = kid + 1 < nk ? offs_at(first[t] + kid + 1) : end[t];
                    const uint32_t g = ((far >> kid) & 1u) + ((far3 >> kid) & 1u);
                    if (g && hi > lo) f(first[t] | kid, g, lo, hi - lo, ((gi * 3u + (uint32_t)t) << d) | kid);
                    lo = hi;
                }
            } else {
                // d > 4: one child at a time
                uint32_t lo = lo0[t];
                for (uint32_t kid = 0; kid < nk; ++kid) {
                    const uint32_t hi = kid + 1 < nk ? offs_at(first[t] + kid + 1) : end[t];
                    uint32_t linf = 0;
#pragma unroll
                    for (int k = 0; k < DM; ++k) {
                        if (k >= d) break;
                        const uint32_t pos =
                            2u * (uint32_t)(ek[k] + 1) + ((kid >> (d - 1 - k)) & 1u);
                        const uint32_t dk = (dist[k] >> (3u * pos)) & 7u;
                        linf = dk > linf ? dk : linf;
                    }
                    if (linf > 1 && hi > lo) f(first[t] | kid, linf - 1, lo, hi - lo, ((gi * 3u + (uint32_t)t) << d) | kid);
                    lo = hi;
                }
            }
        }
    }
}

// Type-II entries (thread per (row, bucket j)): the per-gap totals of the partner
// sets, draw 0 of each single-chunk stream (most streams end there), and for the
// remaining streams a descriptor plus their partner segments in rank order.  A
// partner set whose sorted positions continue those of the previous set of the
// same gap extends its segment (the index-to-vertex map is the same), so the
// children of a parent neighbour that share a gap usually form one segment.
template <int DIM>
__global__ void __launch_bounds__(kEnumThreads, 4) k_enum2(DevCfg cfg) {
    const int lane = threadIdx.x & 31;
    const int d = DIM ? DIM : cfg.d;
    Counters C;
    unsigned long long t2_items_local = 0;
    unsigned int count = *cfg.ent2_count < cfg.ent2_cap ? *cfg.ent2_count : cfg.ent2_cap;
    if (count > cfg.ent2_hi) count = cfg.ent2_hi;
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int b0 = cfg.ent2_lo + blockIdx.x * blockDim.x; b0 < count; b0 += stride) {
        const unsigned int q = b0 + threadIdx.x;
        const bool active = q < count;
        EntryCtx x;
        // per gap: partner cells, segments, total size, end of the last segment
        uint32_t cnt[2] = {0u, 0u}, nseg[2] = {0u, 0u}, sum[2] = {0u, 0u}, keep[2] = {0u, 0u};
        uint32_t s0[2], tidx[2], pack[2] = {0u, 0u};
        // d = 2: the ranks (< 36) of the partner cells visited, per gap, so that the
        // second visit below goes straight to them
        unsigned long long vis0 = 0ull, vis1 = 0ull;
        if (active) {
            x = decode_entry<DIM>(cfg, cfg.ent2[q], d, false);
            uint32_t nxt[2] = {0xffffffffu, 0xffffffffu};
            auto add = [&](int gi, uint32_t lo, uint32_t len) {
                cnt[gi] += 1u;
                nseg[gi] += lo != nxt[gi] ? 1u : 0u;
                sum[gi] += len;
                nxt[gi] = lo + len;
            };
            for_partners<DIM>(cfg, x, d,
                              [&](uint32_t, uint32_t g, uint32_t lo, uint32_t len, uint32_t rank) {
                                  if (g == 1) {
                                      add(0, lo, len);
                                      if (DIM == 2) vis0 |= 1ull << rank;
                                  } else {
                                      add(1, lo, len);
                                      if (DIM == 2) vis1 |= 1ull << rank;
                                  }
                              });
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                s0[g] = 0xffffffffu;
                if (!cnt[g]) continue;
                t2_items_local += cnt[g];
                pack[g] = (uint32_t)x.l | ((uint32_t)x.i << 5) | ((uint32_t)x.j << 11) |
                          ((uint32_t)g << 17) | (kTagJump << 18);
                tidx[g] = ((((uint32_t)x.i * cfg.L + x.j) * (cfg.lcap + 1) + x.l) << 1) + g;
                const TwoEntry te = cfg.tii[tidx[g]];
                const unsigned long long tot = (unsigned long long)x.a_len * sum[g];
                keep[g] = 1u;
                if (tot <= (1ull << te.k)) {
                    // draw 0 when single precision decides it; otherwise (inside the
                    // band, or in FP64 mode) the stream is kept whole and the sampling
                    // kernel takes the same draw with its exact rule
                    const P4 o = philox(x.A, pack[g], 0u, 0u, cfg.seed_lo, cfg.seed_hi);
                    unsigned long long X = 0;
                    int rj = 2;
                    if (te.one)
                        rj = tot == 0 ? 0 : 1;
                    else if (cfg.precision == 0)
                        rj = jump32(o.x, o.y, te.invLb, tot, &X);
                    if (rj != 2) {
                        ++C.draws;
                        if (rj == 0)
                            keep[g] = 0u;
                        else
                            s0[g] = (uint32_t)X;
                    }
                }
            }
        }
        // one atomic per block for the streams and one for their segments
        const uint32_t nst = keep[0] + keep[1];
        const uint32_t nsg = (keep[0] ? nseg[0] : 0u) + (keep[1] ? nseg[1] : 0u);
        const uint32_t want[2] = {nst, nsg};
        unsigned long long* const ctr[2] = {cfg.stream_count, cfg.seg_count};
        unsigned long long slot[2];
        block_alloc<2>(want, ctr, slot);
        unsigned long long st_base = slot[0], sg_base = slot[1];
        if (nst && !cfg.count_only) {
            unsigned long long off[2];
            uint32_t pos[2] = {0u, 0u}, pre[2] = {0u, 0u}, nxt[2] = {0xffffffffu, 0xffffffffu};
            off[0] = sg_base;
            off[1] = sg_base + (keep[0] ? nseg[0] : 0u);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (!keep[g]) continue;
                if (st_base < cfg.stream_cap) {
                    // chunks of 2^k indices; a stream needing 2^32 or more is an error
                    const TwoEntry te = cfg.tii[tidx[g]];
                    const int k = te.k;
                    const unsigned long long tot = (unsigned long long)x.a_len * sum[g];
                    unsigned long long nch = (tot + (1ull << k) - 1) >> k;
                    if (nch > 0xffffffffull) {
                        atomicOr(cfg.error, 1u);
                        nch = 1;
                    }
                    cfg.stream_chunks[st_base] = (uint32_t)nch;
                    Stream st;
                    st.A = x.A;
                    st.pack = pack[g];
                    st.a_begin = x.a_lo;
                    st.a_len = x.a_len;
                    st.seg_off = (uint32_t)off[g];  // < seg_cap <= 2^32 when kept
                    st.seg_cnt = nseg[g];
                    st.S = sum[g];
                    st.tii = tidx[g];
                    st.s0 = s0[g];
                    st.invLb = te.invLb;
                    st.log2pbar = te.log2pbar;
                    st.kone = (uint32_t)te.k | (te.one ? 0x100u : 0u);
                    cfg.streams[st_base] = st;
                }
                ++st_base;
            }
            auto put = [&](int gi, uint32_t lo, uint32_t len) {
                if (!keep[gi]) return;
                if (lo != nxt[gi]) {
                    const unsigned long long at = off[gi] + pos[gi];
                    if (at < cfg.seg_cap) cfg.segs[at] = Seg{lo, pre[gi]};
                    pos[gi] += 1u;
                }
                pre[gi] += len;
                nxt[gi] = lo + len;
            };
            if constexpr (DIM == 2) {
                // the visited cells again, in rank order: the parent neighbour of digits
                // (e0, e1) = (p / 3 - 1, p % 3 - 1), child kid, offsets from cache
                const uint32_t PA = x.A >> 2;
                const int lev = x.l - 1;
                const uint32_t m0 = dim_mask(2, 0, lev), m1 = dim_mask(2, 1, lev);
                const uint32_t a0 = dil_add(PA, m0, 2u, -1), b0 = PA & m0, c0 = dil_add(PA, m0, 2u, 1);
                const uint32_t a1 = dil_add(PA, m1, 1u, -1), b1 = PA & m1, c1 = dil_add(PA, m1, 1u, 1);
#pragma unroll
                for (int gi = 0; gi < 2; ++gi) {
                    if (!keep[gi]) continue;
                    unsigned long long m = gi == 0 ? vis0 : vis1;
                    while (m) {
                        const uint32_t rank = (uint32_t)__ffsll((long long)m) - 1u;
                        m &= m - 1ull;
                        const uint32_t pidx = rank >> 2, kid = rank & 3u;
                        const uint32_t e0 = pidx / 3u, e1 = pidx - 3u * e0;
                        const uint32_t P0 = e0 == 0u ? a0 : (e0 == 1u ? b0 : c0);
                        const uint32_t P1 = e1 == 0u ? a1 : (e1 == 1u ? b1 : c1);
                        const uint32_t cell = ((P0 | P1) << 2) | kid;
                        const uint32_t lo = cfg.offs[x.baseB + (uint32_t)((uint64_t)cell << x.sB)];
                        const uint32_t hi =
                            cfg.offs[x.baseB + (uint32_t)(((uint64_t)cell + 1) << x.sB)];
                        put(gi, lo, hi - lo);
                    }
                }
            } else {
                for_partners<DIM>(cfg, x, d, [&](uint32_t, uint32_t g, uint32_t lo, uint32_t len,
                                                 uint32_t) {
                    if (g == 1)
                        put(0, lo, len);
                    else
                        put(1, lo, len);
                });
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) t2_items_local += __shfl_down_sync(0xffffffffu, t2_items_local, o);
    if (lane == 0 && t2_items_local) atomicAdd(&cfg.stats[kStatT2Items], t2_items_local);
    flush_counters(cfg, C);
}

// Visit the neighbour cells B of A on level l (B >= A when j = i) that hold a
// vertex of bucket j: f(B, lo, len) with the range of sorted positions (len > 0),
// in the order of the offset index (digits e_k + 1, dimension 0 most significant).
// The neighbours go in groups of three that differ in the last digit only; the
// offsets of a group are loaded together.
template <int DIM, class F>
__device__ __forceinline__ void for_neighbours(const DevCfg& cfg, const EntryCtx& x, int d, F f) {
    constexpr int DM = DIM ? DIM : kMaxDim;
    constexpr uint32_t NG = DIM == 1 ? 1u : DIM == 2 ? 3u : DIM == 3 ? 9u : DIM == 4 ? 27u : 0u;
    uint32_t ng = NG;
    if (DIM == 0) {
        ng = 1;
        for (int k = 1; k < d; ++k) ng *= 3u;
    }
    const bool same = x.j == x.i;
    uint32_t am[DM], a0[DM], ap[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
        if (k >= d) break;
        const uint32_t mask = dim_mask(d, k, x.l), unit = 1u << (d - 1 - k);
        am[k] = dil_add(x.A, mask, unit, -1);
        a0[k] = x.A & mask;
        ap[k] = dil_add(x.A, mask, unit, 1);
    }
    const int kl = d - 1;
#pragma unroll(DIM == 1 || DIM == 2 ? NG : 1)
    for (uint32_t gi = 0; gi < ng; ++gi) {
        uint32_t q = gi, Bg = 0;
        bool okg = true;
#pragma unroll
        for (int k = DM - 1; k >= 0; --k) {
            if (k >= kl) continue;
            const int e = (int)(q % 3u) - 1;
            q /= 3u;
            okg = okg && digit_ok(e, x.l);
            Bg |= e < 0 ? am[k] : e > 0 ? ap[k] : a0[k];
        }
        if (!okg) continue;
        uint32_t B[3], lo[3], len[3];
        bool use[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int e = t - 1;
            B[t] = Bg | (e < 0 ? am[kl] : e > 0 ? ap[kl] : a0[kl]);
            use[t] = digit_ok(e, x.l) && !(same && B[t] < x.A);
            lo[t] = 0;
            len[t] = 0;
            if (use[t]) range_of(cfg, x, B[t], &lo[t], &len[t]);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (use[t] && len[t]) f(B[t], lo[t], len[t]);
    }
}

// Type-I entries (thread per (row, bucket j)): every non-empty neighbour cell B
// of A (B >= A when j = i) gives an item V_i^A x V_j^B, split into sub-items of at
// most kSplitAB pairs.
template <int DIM>
__global__ void __launch_bounds__(kEnumThreads) k_enum1(DevCfg cfg) {
    const int lane = threadIdx.x & 31;
    const int d = DIM ? DIM : cfg.d;
    unsigned long long t1_items_local = 0, t1_refs_local = 0;
    unsigned int count = *cfg.ent1_count < cfg.ent1_cap ? *cfg.ent1_count : cfg.ent1_cap;
    if (count > cfg.ent1_hi) count = cfg.ent1_hi;
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int b0 = cfg.ent1_lo + blockIdx.x * blockDim.x; b0 < count; b0 += stride) {
        const unsigned int q = b0 + threadIdx.x;
        const bool active = q < count;
        EntryCtx x;
        if (active) x = decode_entry<DIM>(cfg, cfg.ent1[q], d, true);
        // sub-items: a-chunks of ac = kSplitAB / bc rows (>= 4) times b-chunks of
        // bc = min(b_len, kSplitB) columns, ceil(b_len / kSplitB) of them
        auto split = [&](uint32_t b_len, uint32_t* ac, uint32_t* bc, uint32_t* na) {
            *bc = b_len < kSplitB ? b_len : kSplitB;
            *ac = udiv24(kSplitAB, *bc);
            const uint32_t num = x.a_len + *ac - 1;
            *na = num < (1u << 24) ? udiv24(num, *ac) : num / *ac;
            return *na * ((b_len + kSplitB - 1) / kSplitB);
        };
        uint32_t nsub = 0;
        if (active) {
            for_neighbours<DIM>(cfg, x, d, [&](uint32_t, uint32_t, uint32_t len) {
                uint32_t ac, bc, na;
                nsub += split(len, &ac, &bc, &na);
            });
        }
        const uint32_t want[1] = {nsub};
        unsigned long long* const ctr[1] = {cfg.t1_count};
        unsigned long long slot[1];
        block_alloc<1>(want, ctr, slot);
        unsigned long long tbase = slot[0];
        if (nsub && !cfg.count_only) {
            for_neighbours<DIM>(cfg, x, d, [&](uint32_t B, uint32_t lo, uint32_t len) {
                uint32_t ac, bc, na;
                split(len, &ac, &bc, &na);
                const uint32_t tri = (B == x.A && x.j == x.i) ? 0x80000000u : 0u;
                for (uint32_t ya = 0; ya < x.a_len; ya += ac) {
                    for (uint32_t yb = 0; yb < len; yb += bc, ++tbase) {
                        if (tbase < cfg.t1_cap) {
                            T1Item it;
                            it.a_begin = x.a_lo + ya;
                            it.a_len = (x.a_len - ya) < ac ? (x.a_len - ya) : ac;
                            it.b_begin = lo + yb;
                            const uint32_t blen = (len - yb) < bc ? (len - yb) : bc;
                            it.b_len = blen | tri;
                            cfg.t1[tbase] = it;
                            cfg.t1_pairs[tbase] = it.a_len * blen;
                        }
                    }
                }
                // every a-chunk meets every b-chunk: sum of side lengths over sub-items
                t1_refs_local += (unsigned long long)x.a_len * ((len + kSplitB - 1) / kSplitB) +
                                 (unsigned long long)len * na;
            });
            t1_items_local += nsub;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        t1_items_local += __shfl_down_sync(0xffffffffu, t1_items_local, o);
        t1_refs_local += __shfl_down_sync(0xffffffffu, t1_refs_local, o);
    }
    if (lane == 0 && t1_items_local) {
        atomicAdd(&cfg.stats[kStatT1Items], t1_items_local);
        atomicAdd(&cfg.stats[kStatT1VertexRefs], t1_refs_local);
    }
}

// ------------------------------------------------------------------ balanced work
// Largest q in [0, nq) with pre[q] <= f, for a nondecreasing prefix with
// pre[0] <= f < pre[nq]: a 32-way search in which the lanes test 32 pivots at
// once, so about log_32(nq) dependent loads.  All lanes return the same q.
__device__ __forceinline__ uint32_t warp_search(const unsigned long long* pre, uint32_t nq,
                                                unsigned long long f) {
    const int lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = nq;  // pre[lo] <= f < pre[hi]
    while (hi - lo > 1) {
        const uint32_t span = hi - lo;
        const uint32_t piv = lo + (uint32_t)(((unsigned long long)span * (uint32_t)(lane + 1)) >> 5);
        const bool ok = piv < hi && pre[piv] <= f;
        const int k = __popc(__ballot_sync(0xffffffffu, ok));  // pivots 0 .. k-1 are <= f
        const uint32_t nlo = __shfl_sync(0xffffffffu, piv, k > 0 ? k - 1 : 0);
        const uint32_t nhi = __shfl_sync(0xffffffffu, piv, k < 31 ? k : 31);
        if (k > 0) lo = nlo;
        hi = nhi;
    }
    return lo;
}

// For each lane: the largest j in [0, 31] with v_j <= f, where v_j is lane j's
// value, v is nondecreasing in the lane index and v_0 <= f.
__device__ __forceinline__ int warp_last_le(unsigned long long v, unsigned long long f) {
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const unsigned long long x = __shfl_sync(0xffffffffu, v, j + step);
        if (x <= f) j += step;
    }
    return j;
}

// The same for 32-bit signed values.
__device__ __forceinline__ int warp_last_le32(int v, int f) {
    int j = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int x = __shfl_sync(0xffffffffu, v, j + step);
        if (x <= f) j += step;
    }
    return j;
}

// ------------------------------------------------------------------ type I
// Every pair of every type-I item (Algorithm 1: "emit each edge with p_uv").  The
// pairs of all items form one index space through the exclusive prefix t1_pre;
// a warp takes kT1Grab consecutive pairs at a time, so all warps end together
// whatever the item sizes.  A round tests up to 32 kT1Pairs consecutive pairs, lane f
// the pairs f0 + f, f0 + 32 + f, ... (independent chains of loads and Philox rounds
// per lane), each finding its item in a window of 32 consecutive items held one
// per lane; the window starts at the item of f0 and the round stops at the end
// of the window's last item.
constexpr int kT1Threads = 256;
constexpr unsigned kT1Grab = 1024;
constexpr int kT1Pairs = 2;  // pairs per lane and round

// HRG: the HRG instantiation (d = 1; its own registers, so that the GIRG d = 1 kernel
// keeps the budget of its own decisions).
template <int DIM, bool HRG = false>
__device__ __forceinline__ void type1_loop(const DevCfg& cfg, const View& V, WarpEdges& we,
                                           Counters& C) {
    const int lane = threadIdx.x & 31;
    const uint32_t nit = (uint32_t)(*cfg.t1_count < cfg.t1_cap ? *cfg.t1_count : cfg.t1_cap);
    const unsigned long long* pre = cfg.t1_pre;
    const unsigned long long total = pre[nit];
    uint32_t t1_edges = 0;
    for (;;) {
        unsigned long long F0 = 0;
        if (lane == 0) F0 = atomicAdd(&cfg.work64[0], (unsigned long long)kT1Grab);
        F0 = __shfl_sync(0xffffffffu, F0, 0);
        if (F0 >= total) break;
        // pair indices relative to F0: an item holds at most kSplitAB pairs, so the
        // 32 items of a window lie within (-2^13, 2^18) of F0
        const int F1 = (int)(total - F0 < kT1Grab ? total - F0 : kT1Grab);
        uint32_t k = warp_search(pre, nit, F0), wk = 0xffffffffu;
        int wpre = 0, wend = 0;
        T1Item wit{0u, 0u, 0u, 0u};
        for (int f0 = 0; f0 < F1;) {
            if (k != wk) {  // window: items k .. k + 31 with their first and end pairs
                const uint32_t q = k + (uint32_t)lane;
                wpre = q <= nit ? (int)(long long)(pre[q] - F0) : 0x7fffffff;
                wend = q < nit ? (int)(long long)(pre[q + 1] - F0) : 0x7fffffff;
                if (q < nit) wit = cfg.t1[q];
                wk = k;
            }
            // the round: pairs [f0, fe), at most 64 and inside the window; lane l takes
            // pairs f0 + l and f0 + 32 + l
            const int wlast = __shfl_sync(0xffffffffu, wend, 31);
            int fe = f0 + 32 * kT1Pairs;
            if (fe > wlast) fe = wlast;
            if (fe > F1) fe = F1;
            bool ok[kT1Pairs];
            uint32_t pu[kT1Pairs], pv[kT1Pairs];
#pragma unroll
            for (int h = 0; h < kT1Pairs; ++h) {
                const int f = f0 + 32 * h + lane;
                const int j = warp_last_le32(wpre, f);
                const uint32_t a_begin = __shfl_sync(0xffffffffu, wit.a_begin, j);
                const uint32_t b_begin = __shfl_sync(0xffffffffu, wit.b_begin, j);
                const uint32_t b_len = __shfl_sync(0xffffffffu, wit.b_len, j);
                const int pj = __shfl_sync(0xffffffffu, wpre, j);
                ok[h] = false;
                pu[h] = 0;
                pv[h] = 0;
                if (f < fe) {
                    const uint32_t bl = b_len & 0x7fffffffu;
                    const uint32_t rr = (uint32_t)(f - pj);
                    // rr / bl from a float reciprocal (rr < 2^24), corrected to the exact quotient
                    uint32_t ia = __float2uint_rz(__uint2float_rn(rr) * __frcp_rn((float)bl));
                    int ib = (int)rr - (int)(ia * bl);
                    if (ib < 0) {
                        --ia;
                        ib += (int)bl;
                    } else if (ib >= (int)bl) {
                        ++ia;
                        ib -= (int)bl;
                    }
                    pu[h] = a_begin + ia;
                    pv[h] = b_begin + (uint32_t)ib;
                    ok[h] = !((b_len & 0x80000000u) && pv[h] <= pu[h]);
                    if (ok[h]) ++C.t1pairs;
                }
            }
            bool edge[kT1Pairs];
            uint32_t ia_id[kT1Pairs], ib_id[kT1Pairs];
#pragma unroll
            for (int h = 0; h < kT1Pairs; ++h) {
                edge[h] = false;
                ia_id[h] = ib_id[h] = 0u;
            }
            if constexpr (HRG) {
                if (cfg.precision == 0) {
                    decide_t1_hrg_xp<kT1Pairs>(cfg, V, ok, pu, pv, C, edge, ia_id, ib_id);
                } else {
#pragma unroll
                    for (int h = 0; h < kT1Pairs; ++h)
                        if (ok[h]) edge[h] = decide_t1<DIM>(cfg, V, pu[h], pv[h], C, &ia_id[h], &ib_id[h]);
                }
            } else if constexpr (DIM >= 1 && DIM <= 4) {
                if (cfg.model == 0 && cfg.precision == 0 && V.rec) {
                    decide_t1_xp<DIM, kT1Pairs>(cfg, V, ok, pu, pv, C, edge, ia_id, ib_id);
                } else {
#pragma unroll
                    for (int h = 0; h < kT1Pairs; ++h)
                        if (ok[h]) edge[h] = decide_t1<DIM>(cfg, V, pu[h], pv[h], C, &ia_id[h], &ib_id[h]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < kT1Pairs; ++h)
                    if (ok[h]) edge[h] = decide_t1<DIM>(cfg, V, pu[h], pv[h], C, &ia_id[h], &ib_id[h]);
            }
#pragma unroll
            for (int h = 0; h < kT1Pairs; ++h) {
                if (edge[h]) {
                    push_edge(cfg, we, ia_id[h], ib_id[h]);
                    ++t1_edges;
                }
            }
            flush_edges<true>(cfg, we, kEdgeBuf - 32 * kT1Pairs);
            // the next round starts in the first item that ends after fe
            f0 = fe;
            k += (uint32_t)__popc(__ballot_sync(0xffffffffu, wend <= fe));
        }
    }
    flush_edges<true>(cfg, we, 1);
    flush_mix(cfg, we);
    unsigned long long te = t1_edges;
    for (int o = 16; o > 0; o >>= 1) te += __shfl_down_sync(0xffffffffu, te, o);
    if (lane == 0 && te) atomicAdd(&cfg.stats[kStatT1Edges], te);
}

template <int DIM, bool HRG = false>
__global__ void __launch_bounds__(kT1Threads, 4) k_type1(DevCfg cfg) {
    if (cfg.lists_ok && *cfg.lists_ok == 0u) return;  // a list overflowed: the round is redone
    __shared__ uint32_t s_ea[kWarps][kEdgeBuf], s_eb[kWarps][kEdgeBuf];
    __shared__ unsigned int s_en[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_en[warp] = 0;
    __syncwarp();
    WarpEdges we{s_ea[warp], s_eb[warp], &s_en[warp]};
    Counters C;
    type1_loop<DIM, HRG>(cfg, sorted_view(cfg), we, C);
    flush_counters(cfg, C);
}

// ------------------------------------------------------------------ type II
// Geometric jumps (Sec. 3.2) over every chunk of every type-II stream: chunk h of
// a stream covers indices [h 2^k, min((h + 1) 2^k, a S)) of its index space
// idx = a S + b (a in V_i^A, b in the concatenated partner sets), and draw t of
// the chunk is Philox of (A, pack, h, t): words 0, 1 give the jump, words 2, 3
// the acceptance U' pbar < p_uv.  Single-chunk streams whose draw 0 the
// enumeration already took resume at draw 1 with its candidate s0.
//
// A lane works one chunk at a time and draws once per round; a lane whose chunk
// ended takes the next chunk of the warp's bundle (32 consecutive chunks of the
// global chunk space, fetched with one atomic and mapped to streams with one
// warp search), so the lanes stay busy however unequal the chunks are.
constexpr int kT2Threads = 256;
constexpr int kT2RefillMin = 8;  // refill idle lanes once this many are idle

template <int DIM, bool HRG = false>
__device__ __forceinline__ void type2_loop(const DevCfg& cfg, const View& V, WarpEdges& we,
                                           Counters& C) {
    const int lane = threadIdx.x & 31;
    const uint32_t nst =
        (uint32_t)(*cfg.stream_count < cfg.stream_cap ? *cfg.stream_count : cfg.stream_cap);
    const unsigned long long* pre = cfg.chunk_pre;
    const unsigned long long total = pre[nst];
    // the warp's bundle: lane j holds stream and chunk index of bundle chunk j
    uint32_t bq = 0, bh = 0;
    int bn = 0, bcur = 0;
    bool drained = false;
    // the lane's chunk
    bool live = false, resumed = false;
    Stream st{};
    TwoFast e{};
    uint32_t h = 0, t = 0;
    long long s = -1;
    unsigned long long start = 0, len = 0;
    bool small = true;  // index space below 2^32
    for (;;) {
        uint32_t idle = __ballot_sync(0xffffffffu, !live);
        if (__popc(idle) >= kT2RefillMin || idle == 0xffffffffu) {
            while (idle) {
                if (bcur == bn) {
                    if (drained) break;
                    unsigned long long g0 = 0;
                    if (lane == 0) g0 = atomicAdd(&cfg.work64[1], 32ull);
                    g0 = __shfl_sync(0xffffffffu, g0, 0);
                    if (g0 >= total) {
                        drained = true;
                        break;
                    }
                    if (g0 + 32 >= total) drained = true;
                    // streams q0 .. q0 + 31 hold the bundle (every stream has a chunk)
                    const uint32_t q0 = warp_search(pre, nst, g0);
                    const uint32_t qw = q0 + (uint32_t)lane;
                    const unsigned long long v = qw <= nst ? pre[qw] : ~0ull;
                    const unsigned long long g = g0 + (unsigned long long)lane;
                    const int j = warp_last_le(v, g);
                    const unsigned long long base = __shfl_sync(0xffffffffu, v, j);
                    bq = q0 + (uint32_t)j;
                    bh = (uint32_t)(g - base);
                    bn = (int)(total - g0 < 32ull ? total - g0 : 32ull);
                    bcur = 0;
                }
                const int nidle = __popc(idle);
                const int take = nidle < bn - bcur ? nidle : bn - bcur;
                const int r = __popc(idle & lanemask_lt());
                const int src = (bcur + r) & 31;
                const uint32_t q = __shfl_sync(0xffffffffu, bq, src);
                const uint32_t hh = __shfl_sync(0xffffffffu, bh, src);
                if (((idle >> lane) & 1u) && r < take) {
                    st = cfg.streams[q];
                    e = TwoFast{st.invLb, st.log2pbar, st.tii, (st.kone >> 8) != 0u};
                    const int kc = (int)(st.kone & 0xffu);
                    const unsigned long long tot = (unsigned long long)st.a_len * st.S;
                    small = tot <= 0xffffffffull;
                    h = hh;
                    start = (unsigned long long)h << kc;
                    len = tot - start < (1ull << kc) ? tot - start : (1ull << kc);
                    t = 0;
                    s = -1;
                    resumed = st.s0 != 0xffffffffu;
                    live = true;
                }
                bcur += take;
                idle = __ballot_sync(0xffffffffu, !live);
            }
        }
        if (!__any_sync(0xffffffffu, live)) {
            if (drained && bcur == bn) break;
            continue;
        }
        bool edge = false;
        uint32_t pu = 0, pv = 0, idu = 0, idv = 0;
        if (live) {
            const P4 o = philox(st.A, st.pack, h, t, cfg.seed_lo, cfg.seed_hi);
            bool cand = true;
            if (t == 0 && resumed) {
                s = (long long)st.s0;
            } else {
                ++C.draws;
                unsigned long long X;
                if (draw_jump_fast(cfg, e, o, len - (unsigned long long)(s + 1), &X, C) == 0) {
                    live = false;
                    cand = false;
                } else {
                    s += 1 + (long long)X;
                }
            }
            ++t;
            if (cand) {
                ++C.cands;
                const unsigned long long idx = start + (unsigned long long)s;
                uint32_t ia, ib;
                if (idx < (1ull << 24)) {
                    // idx / S from a float reciprocal (exact to one unit below 2^24)
                    const uint32_t ix = (uint32_t)idx;
                    ia = __float2uint_rz(__uint2float_rn(ix) * __frcp_rn((float)st.S));
                    int r = (int)ix - (int)(ia * st.S);
                    if (r < 0) {
                        --ia;
                        r += (int)st.S;
                    } else if (r >= (int)st.S) {
                        ++ia;
                        r -= (int)st.S;
                    }
                    ib = (uint32_t)r;
                } else if (small) {
                    ia = (uint32_t)idx / st.S;
                    ib = (uint32_t)idx - ia * st.S;
                } else {
                    ia = (uint32_t)(idx / st.S);
                    ib = (uint32_t)(idx - (unsigned long long)ia * st.S);
                }
                // the last partner set with pre <= ib: up to 4 segments loaded at once
                // (one dependent load), else a binary search
                const Seg* sp = cfg.segs + st.seg_off;
                Seg sg;
                if (st.seg_cnt <= 4) {
                    Seg s1{0u, 0xffffffffu}, s2{0u, 0xffffffffu}, s3{0u, 0xffffffffu};
                    sg = sp[0];
                    if (st.seg_cnt > 1) s1 = sp[1];
                    if (st.seg_cnt > 2) s2 = sp[2];
                    if (st.seg_cnt > 3) s3 = sp[3];
                    if (s1.pre <= ib) sg = s1;
                    if (s2.pre <= ib) sg = s2;
                    if (s3.pre <= ib) sg = s3;
                } else {
                    uint32_t lo = 0, hi = st.seg_cnt;
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (sp[mid].pre <= ib) lo = mid; else hi = mid;
                    }
                    sg = sp[lo];
                }
                pu = st.a_begin + ia;
                pv = sg.b_begin + (ib - sg.pre);
                edge = accept_t2_fast<DIM, HRG>(cfg, V, pu, pv, o.z, o.w, e, C, &idu, &idv);
            }
        }
        if (edge) push_edge(cfg, we, idu, idv);
        flush_edges(cfg, we, kEdgeBuf - 32);
    }
    flush_edges(cfg, we, 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&cfg.stats[kStatT2Chunks], total);
}

template <int DIM, bool HRG = false>
__global__ void __launch_bounds__(kT2Threads, 4) k_type2(DevCfg cfg) {
    if (cfg.lists_ok && *cfg.lists_ok == 0u) return;  // a list overflowed: the round is redone
    __shared__ uint32_t s_ea[kWarps][kEdgeBuf], s_eb[kWarps][kEdgeBuf];
    __shared__ unsigned int s_en[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_en[warp] = 0;
    __syncwarp();
    WarpEdges we{s_ea[warp], s_eb[warp], &s_en[warp]};
    Counters C;
    type2_loop<DIM, HRG>(cfg, sorted_view(cfg), we, C);
    flush_counters(cfg, C);
}

// ------------------------------------------------------------------ all pairs
// Every pair u < v of the original order (Table 1, "Pairwise"): tiles of
// 64 x 64 vertices, upper triangle only.
template <int DIM>
__global__ void __launch_bounds__(256) k_allpairs(DevCfg cfg, View V, unsigned int ntile) {
    __shared__ uint32_t s_ea[kWarps][kEdgeBuf], s_eb[kWarps][kEdgeBuf];
    __shared__ unsigned int s_en[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_en[warp] = 0;
    __syncwarp();
    WarpEdges we{s_ea[warp], s_eb[warp], &s_en[warp]};
    Counters C;
    const unsigned long long ntri = (unsigned long long)ntile * (ntile + 1) / 2;
    for (unsigned long long t = blockIdx.x; t < ntri; t += gridDim.x) {
        // tile (tu, tv), tu <= tv, from the triangular index t (integer search)
        unsigned int lo = 0, hi = ntile;  // largest tv with tv (tv + 1) / 2 <= t
        while (hi - lo > 1) {
            const unsigned int mid = (lo + hi) >> 1;
            if ((unsigned long long)mid * (mid + 1) / 2 <= t) lo = mid; else hi = mid;
        }
        const unsigned int tv = lo;
        const unsigned int tu = (unsigned int)(t - (unsigned long long)tv * (tv + 1) / 2);
        for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
            const uint32_t u = tu * 64 + (q >> 6), v = tv * 64 + (q & 63);
            bool edge = false;
            uint32_t a = 0, b = 0;
            if (u < v && v < (uint32_t)V.n) edge = decide_t1<DIM>(cfg, V, u, v, C, &a, &b);
            if (edge) push_edge(cfg, we, a, b);
            flush_edges(cfg, we, kEdgeBuf - 32);
        }
    }
    flush_edges(cfg, we, 1);
}

bool det_tables_pairs() { return det_tables_ready(); }

// ------------------------------------------------------------------ launchers
void launch_rows(const DevCfg& cfg, cudaStream_t st) {
    int64_t b = (cfg.n + kAllocThreads - 1) / kAllocThreads;
    if (b > device_sms() * 16) b = device_sms() * 16;
    if (b < 1) b = 1;
    ++g_launches;
    k_rows<<<(unsigned)b, kAllocThreads, 0, st>>>(cfg);
}

__global__ void k_prep_lists(DevCfg cfg, unsigned long long* lens, unsigned int* ok) {
    const unsigned long long c1 = *cfg.t1_count, cs = *cfg.stream_count;
    *ok = c1 <= cfg.t1_cap && cs <= cfg.stream_cap && *cfg.seg_count <= cfg.seg_cap ? 1u : 0u;
    const unsigned long long n1 = c1 < cfg.t1_cap ? c1 : cfg.t1_cap;
    const unsigned long long ns = cs < cfg.stream_cap ? cs : cfg.stream_cap;
    cfg.t1_pairs[n1] = 0u;
    cfg.stream_chunks[ns] = 0u;
    cfg.work64[0] = 0ull;
    cfg.work64[1] = 0ull;
    lens[0] = n1 + 1;
    lens[1] = ns + 1;
}

void launch_prep_lists(const DevCfg& cfg, unsigned long long* lens, unsigned int* ok,
                       cudaStream_t st) {
    ++g_launches;
    k_prep_lists<<<1, 1, 0, st>>>(cfg, lens, ok);
}

void launch_enumerate(const DevCfg& cfg, cudaStream_t st) {
    g_launches += 2;
    const unsigned grid = (unsigned)device_sms() * 8;
    switch (cfg.d) {
        case 1: k_enum2<1><<<grid, kEnumThreads, 0, st>>>(cfg);
                k_enum1<1><<<grid, kEnumThreads, 0, st>>>(cfg); break;
        case 2: k_enum2<2><<<grid, kEnumThreads, 0, st>>>(cfg);
                k_enum1<2><<<grid, kEnumThreads, 0, st>>>(cfg); break;
        case 3: k_enum2<3><<<grid, kEnumThreads, 0, st>>>(cfg);
                k_enum1<3><<<grid, kEnumThreads, 0, st>>>(cfg); break;
        case 4: k_enum2<4><<<grid, kEnumThreads, 0, st>>>(cfg);
                k_enum1<4><<<grid, kEnumThreads, 0, st>>>(cfg); break;
        default: k_enum2<0><<<grid, kEnumThreads, 0, st>>>(cfg);
                 k_enum1<0><<<grid, kEnumThreads, 0, st>>>(cfg); break;
    }
}

// Blocks of a persistent launch: the resident blocks per SM times the SMs.
template <class K>
static unsigned persistent_grid(K kernel, int threads) {
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return (unsigned)(device_sms() * per);
}

void launch_type1(const DevCfg& cfg, cudaStream_t st) {
    ++g_launches;
    if (cfg.model == 1) {  // HRG (d = 1)
        static const unsigned grid = persistent_grid(k_type1<1, true>, kT1Threads);
        k_type1<1, true><<<grid, kT1Threads, 0, st>>>(cfg);
        return;
    }
    switch (cfg.d) {
#define GG_T1(D)                                                                     \
    {                                                                                \
        static const unsigned grid = persistent_grid(k_type1<D>, kT1Threads);        \
        k_type1<D><<<grid, kT1Threads, 0, st>>>(cfg);                                \
        break;                                                                       \
    }
        case 1: GG_T1(1)
        case 2: GG_T1(2)
        case 3: GG_T1(3)
        case 4: GG_T1(4)
        default: GG_T1(0)
#undef GG_T1
    }
}

void launch_type2(const DevCfg& cfg, cudaStream_t st) {
    ++g_launches;
    if (cfg.model == 1) {  // HRG (d = 1)
        static const unsigned grid = persistent_grid(k_type2<1, true>, kT2Threads);
        k_type2<1, true><<<grid, kT2Threads, 0, st>>>(cfg);
        return;
    }
    switch (cfg.d) {
#define GG_T2(D)                                                                     \
    {                                                                                \
        static const unsigned grid = persistent_grid(k_type2<D>, kT2Threads);        \
        k_type2<D><<<grid, kT2Threads, 0, st>>>(cfg);                                \
        break;                                                                       \
    }
        case 1: GG_T2(1)
        case 2: GG_T2(2)
        case 3: GG_T2(3)
        case 4: GG_T2(4)
        default: GG_T2(0)
#undef GG_T2
    }
}

void launch_allpairs(const DevCfg& cfg, const uint32_t* X, const double* w, const float* sv,
                     cudaStream_t st) {
    View V{X, sv, w, nullptr, nullptr, nullptr, nullptr, cfg.n, nullptr};
    const unsigned int ntile = (unsigned int)((cfg.n + 63) / 64);
    unsigned long long ntri = (unsigned long long)ntile * (ntile + 1) / 2;
    const unsigned int gmax = (unsigned int)device_sms() * 8;
    unsigned int grid = ntri < gmax ? (unsigned int)ntri : gmax;
    ++g_launches;
    switch (cfg.d) {
        case 1: k_allpairs<1><<<grid, 256, 0, st>>>(cfg, V, ntile); break;
        case 2: k_allpairs<2><<<grid, 256, 0, st>>>(cfg, V, ntile); break;
        case 3: k_allpairs<3><<<grid, 256, 0, st>>>(cfg, V, ntile); break;
        case 4: k_allpairs<4><<<grid, 256, 0, st>>>(cfg, V, ntile); break;
        default: k_allpairs<0><<<grid, 256, 0, st>>>(cfg, V, ntile); break;
    }
}

}  // namespace gg
