// Expected average degree of a GIRG and the search for its scale (Sec. 4.1, App. B.2).
#include "solver.h"

#include <algorithm>
#include <cmath>
#include <system_error>
#include <thread>

namespace gg {

namespace {

// Chunks [c kChunk, min((c + 1) kChunk, n)) of an index range, handed to up to 16 host
// threads (chunk c to thread c mod threads) when `parallel` (work with an exp or log per
// index; cheaper work does not repay starting the threads), else all on the caller's
// thread.  The chunks do not depend on the thread count, so per-chunk results combined
// in chunk order are the same either way and on every machine.
constexpr size_t kChunk = 16384;

template <class F>
void for_chunks(size_t n, bool parallel, F f) {
    const size_t nc = (n + kChunk - 1) / kChunk;
    size_t nt = 1;
    if (parallel && nc > 1) {  // the core count is read once (a file read on Linux)
        static const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        nt = std::min<size_t>(hw, nc);
    }
    if (nt <= 1) {
        for (size_t c = 0; c < nc; ++c) f(c, c * kChunk, std::min(n, (c + 1) * kChunk));
        return;
    }
    auto run = [&](size_t t) {
        for (size_t c = t; c < nc; c += nt) f(c, c * kChunk, std::min(n, (c + 1) * kChunk));
    };
    std::vector<std::thread> pool;
    std::vector<size_t> mine = {0};  // the caller's share, plus that of any thread not started
    for (size_t t = 1; t < nt; ++t) {
        try {
            pool.emplace_back(run, t);
        } catch (const std::system_error&) {
            mine.push_back(t);
        }
    }
    for (size_t t : mine) run(t);
    for (auto& th : pool) th.join();
}

}  // namespace

void DegreeModel::set_split(double thr, std::vector<double> top, double sw, double s2, double sx,
                            double sx2) {
    thr_ = thr;
    sw_ = sw;
    s2_ = s2;
    sx_ = sx;
    sx2_ = sx2;
    top_ = std::move(top);
    const size_t m = top_.size();
    const bool tp = T_ > 0.0;
    const double inv = tp ? 1.0 / T_ : 0.0;
    mi_ = (tp && inv == std::floor(inv) && inv <= 8.0) ? (int)inv : 0;
    const bool logs = tp && !mi_;  // the log path's arrays; the others stay empty
    suf_.assign(m + 1, 0.0);
    suf2_.assign(m + 1, 0.0);
    b_.assign(logs ? m + 1 : 0, 0.0);
    sr_.assign(logs ? m + 1 : 0, 0.0);
    sr2_.assign(logs ? m + 1 : 0, 0.0);
    py_.assign(mi_ ? m : 0, 0.0);
    spy_.assign(mi_ ? m + 1 : 0, 0.0);
    spy2_.assign(mi_ ? m + 1 : 0, 0.0);
    if (logs) {  // b = log(w) / T and the ratios r_i = e^(b_(i+1) - b_i) <= 1, in parallel
        for_chunks(m, true, [&](size_t, size_t lo, size_t hi) {
            for (size_t i = lo; i < hi; ++i) b_[i] = std::log(top_[i]) / T_;
        });
        for_chunks(m, true, [&](size_t, size_t lo, size_t hi) {
            for (size_t i = lo; i < hi; ++i) sr2_[i] = i + 1 < m ? std::exp(b_[i + 1] - b_[i]) : 0.0;
        });
    }
    for (size_t i = m; i-- > 0;) {  // from the light end
        suf_[i] = suf_[i + 1] + top_[i];
        suf2_[i] = suf2_[i + 1] + top_[i] * top_[i];
        if (mi_) {
            const double y = top_[i] / thr;
            double p = y;
            for (int q = 1; q < mi_; ++q) p *= y;
            py_[i] = p;
            spy_[i] = spy_[i + 1] + p;
            spy2_[i] = spy2_[i + 1] + p * p;
            continue;
        }
        if (logs) {
            const double r = sr2_[i];  // the ratio, replaced by the suffix aggregate
            sr_[i] = 1.0 + r * sr_[i + 1];
            sr2_[i] = 1.0 + r * r * sr2_[i + 1];
        }
    }
}

double DegreeModel::needed_threshold(double K) const {
    const double wmax = top_.empty() ? thr_ : top_[0];
    return W_ / (std::ldexp(K, d_) * wmax);
}

bool DegreeModel::valid(double K) const { return thr_ < needed_threshold(K); }

// Sum over ordered pairs u != v of E[X_uv]: rest x rest, rest x top (both orders), and
// top x top.  In the last, the top vertices u with E_R partners (a prefix of the
// decreasing order, usually a few) and the heaviest one are taken one by one; every
// other u has all other top weights as non-E_R partners, and their sums over such u
// come from the suffix aggregates: sum_u w_u (S - w_u) and sum_u e_u (E - e_u) with
// e = w^(1/T), E = sum e (the self terms are at most half of the products there, as
// every such u has the heaviest vertex as a heavier partner).
double DegreeModel::f(double K, double* slope) const {
    // Every non-E_R pair adds (z - T z^(1/T)) / (1 - T), so K d/dK adds (z - z^(1/T)) /
    // (1 - T): each term below is accumulated as (s1 - T s2) / (1 - T) for f and
    // (s1 - s2) / (1 - T) for the slope K f'(K) (E_R pairs contribute no slope).
    const double T = T_, A = std::ldexp(K, d_) / W_, lA = std::log(A);
    const double lt = std::log(thr_);
    const bool tp = T > 0.0;
    const double inv1mT = tp ? 1.0 / (1.0 - T) : 1.0, lAT = tp ? lA / T : 0.0;
    double val = 0.0, slp = 0.0;
    auto add = [&](double s1, double s2) {  // s2 = 0 when T = 0
        val += (s1 - T * s2) * inv1mT;
        slp += (s1 - s2) * inv1mT;
    };
    // rest x rest
    add(A * (sw_ * sw_ - s2_), tp ? std::exp(lAT + 2.0 * lt / T) * (sx_ * sx_ - sx2_) : 0.0);
    const size_t m = top_.size();
    double C = 0.0;  // (A thr^2)^mi on the integer path
    if (mi_) {
        const double a = A * thr_ * thr_;
        C = a;
        for (int q = 1; q < mi_; ++q) C *= a;
    }
    // top x rest, both orders: sum_u [A w_u sw - T (A w_u thr)^(1/T) sx] / (1 - T)
    {
        const double s1 = A * suf_[0] * sw_;
        double s2 = 0.0;
        if (tp && m) s2 = (mi_ ? C * spy_[0] : std::exp(lAT + lt / T + b_[0]) * sr_[0]) * sx_;
        add(2.0 * s1, 2.0 * s2);
    }
    // top x top: the u with E_R partners one by one (k = their number, non-increasing
    // in u), in chunks of u (in parallel on the exp path) summed in chunk order; u_b is
    // the first u > 0 whose heaviest partner is no E_R partner
    size_t u = 1, ub_hi = m;
    while (u < ub_hi) {  // first u >= 1 with A w_u w_0 < 1 (m if none)
        const size_t mid = u + (ub_hi - u) / 2;
        if (A * top_[mid] * top_[0] < 1.0) ub_hi = mid; else u = mid + 1;
    }
    u = m ? std::max<size_t>(u, 1) : 0;
    const size_t nch = (u + kChunk - 1) / kChunk;
    std::vector<double> cval(nch, 0.0), cslp(nch, 0.0);
    for_chunks(u, tp && !mi_, [&](size_t c, size_t lo, size_t hi) {
        // k at the chunk's first u: the number of v with A w_u w_v >= 1
        size_t k = 0, kh = m;
        {
            const double wu = top_[lo];
            while (k < kh) {
                const size_t mid = k + (kh - k) / 2;
                if (A * wu * top_[mid] < 1.0) kh = mid; else k = mid + 1;
            }
        }
        double v = 0.0, sl = 0.0;
        for (size_t q = lo; q < hi; ++q) {
            const double wu = top_[q];
            while (k > 0 && A * wu * top_[k - 1] < 1.0) --k;
            const size_t k1 = q == k ? k + 1 : k;  // first non-E_R partner
            const double s1 = A * wu * (q > k ? suf_[k] - wu : suf_[k1]);
            double s2 = 0.0;
            if (mi_) {
                s2 = C * py_[q] * spy_[k1];
                if (q > k) s2 -= C * py_[q] * py_[q];  // at most half of the sum
            } else if (tp) {
                const double xu = lAT + b_[q];  // log (A w_u)^(1/T)
                s2 = k1 < m ? std::exp(xu + b_[k1]) * sr_[k1] : 0.0;
                if (q > k) s2 -= std::exp(xu + b_[q]);  // at most half of the sum
            }
            v += (double)k - (q < k ? 1.0 : 0.0);
            v += (s1 - T * s2) * inv1mT;
            sl += (s1 - s2) * inv1mT;
        }
        cval[c] = v;
        cslp[c] = sl;
    });
    for (size_t c = 0; c < nch; ++c) {
        val += cval[c];
        slp += cslp[c];
    }
    if (u < m) {  // u .. m-1: no E_R partners, all other top weights are partners
        const double s1 = A * (suf_[u] * suf_[0] - suf2_[u]);
        double s2 = 0.0;
        if (mi_) {
            s2 = C * (spy_[u] * spy_[0] - spy2_[u]);
        } else if (tp) {
            s2 = std::exp(lAT + b_[u] + b_[0]) *
                 (sr_[u] * sr_[0] - std::exp(b_[u] - b_[0]) * sr2_[u]);
        }
        add(s1, s2);
    }
    if (slope) *slope = slp / (double)n_;
    return val / (double)n_;
}

double DegreeModel::solve(double target, const std::function<void(double)>& fetch) {
    auto eval = [&](double K, double* slope) {
        if (!valid(K)) fetch(0.5 * needed_threshold(K));
        return f(K, slope);
    };
    // start where the sum without E_R capping reaches the target; the capping and the
    // z^(1/T) terms only lower f, so the root lies at or above this K0
    double s2 = s2_;
    for (double w : top_) s2 += w * w;
    const double lead = std::ldexp(1.0, d_) * (W_ * W_ - s2) / (W_ * (T_ > 0.0 ? 1.0 - T_ : 1.0));
    double K0 = target * (double)n_ / lead;
    if (!(K0 > 1e-300 && K0 < 1e300)) K0 = 1.0;
    // Newton on x = ln K with the exact slope K f'(K) > 0 (f is increasing and C^1),
    // safeguarded by the bracket of the iterates seen so far: a step leaving it, or a
    // step longer than ln 4 while one side is open, is replaced by bisection or capped
    const double kMaxStep = std::log(4.0);
    double x = std::log(K0), lo = -HUGE_VAL, hi = HUGE_VAL;
    for (int it = 0; it < 200; ++it) {
        const double K = std::exp(x);
        double slope = 0.0;
        const double g = eval(K, &slope) - target;
        if (std::fabs(g) <= 1e-14 * target) return K;
        if (g < 0.0)
            lo = x;
        else
            hi = x;
        double xn = slope > 0.0 ? x - g / slope : (g < 0.0 ? x + kMaxStep : x - kMaxStep);
        if (lo > -HUGE_VAL && hi < HUGE_VAL) {
            if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
            if (hi - lo <= 1e-14 * std::fabs(hi) + 1e-300) return std::exp(0.5 * (lo + hi));
        } else {
            xn = std::fmin(std::fmax(xn, x - kMaxStep), x + kMaxStep);
        }
        if (std::fabs(xn - x) <= 1e-15 * std::fmax(1.0, std::fabs(x))) return std::exp(xn);
        x = xn;
    }
    return std::exp(x);
}

}  // namespace gg

// ---------------------------------------------------------------- HRG degree
// P(dist < t) for two independent vertices of the hyperbolic disk: radii r with
// density alpha sinh(alpha r) / (cosh(alpha R) - 1), angle difference uniform on
// [0, pi].  For radii r1, r2 the share of angle differences with dist < t is 1 when
// t >= r1 + r2, 0 when t <= |r1 - r2| and otherwise (2/pi) asin(sqrt(s)) with
// s = (cosh t - cosh(r1 - r2)) / (2 sinh r1 sinh r2) (hyperbolic law of cosines).
// The double integral runs in y = R - r over the intervals on which that share is
// smooth; each interval is mapped by y = a + (b - a)(1 - cos u)/2 (which removes
// the square-root behaviour at its ends) and integrated with Gauss-Legendre panels;
// where the share is 1 the radial CDF is used in closed form.
namespace gg {
namespace {

constexpr double kPi = 3.14159265358979323846;

constexpr int kGL = 10;      // Gauss-Legendre points per panel
constexpr int kYPanels = 3;  // panels per smooth y interval
constexpr int kTPanels = 2;  // panels per t interval

struct GaussLegendre {
    double x[kGL], w[kGL];
    GaussLegendre() {
        // roots of P_kGL by Newton's method from Tricomi's initial guesses
        for (int i = 0; i < kGL; ++i) {
            const double th = kPi * (4.0 * (i + 1) - 1.0) / (4.0 * kGL + 2.0);
            double z = std::cos(th), dp = 1.0;
            for (int it = 0; it < 60; ++it) {
                double pk = z, pkm1 = 1.0;  // P_1, P_0
                for (int k = 2; k <= kGL; ++k) {
                    const double pn = ((2 * k - 1) * z * pk - (k - 1) * pkm1) / k;
                    pkm1 = pk;
                    pk = pn;
                }
                dp = kGL * (pkm1 - z * pk) / (1.0 - z * z);
                const double step = pk / dp;
                z -= step;
                if (std::fabs(step) <= 1e-17) break;
            }
            double pk = z, pkm1 = 1.0;
            for (int k = 2; k <= kGL; ++k) {
                const double pn = ((2 * k - 1) * z * pk - (k - 1) * pkm1) / k;
                pkm1 = pk;
                pk = pn;
            }
            dp = kGL * (pkm1 - z * pk) / (1.0 - z * z);
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const GaussLegendre& gl() {
    static const GaussLegendre g;
    return g;
}

// Nodes and weights of int_a^b under y = a + (b - a)(1 - cos u)/2, u in [0, pi].
int cos_mapped_rule(double a, double b, int panels, double* y, double* wt) {
    const GaussLegendre& g = gl();
    int k = 0;
    for (int p = 0; p < panels; ++p) {
        const double u0 = kPi * p / panels, u1 = kPi * (p + 1) / panels;
        const double h = 0.5 * (u1 - u0), m = 0.5 * (u0 + u1);
        for (int i = 0; i < kGL; ++i) {
            const double u = m + h * g.x[i];
            y[k] = a + 0.5 * (b - a) * (1.0 - std::cos(u));
            wt[k] = h * g.w[i] * 0.5 * (b - a) * std::sin(u);
            ++k;
        }
    }
    return k;
}

struct Disk {
    double alpha, R, cm1;  // cm1 = cosh(alpha R) - 1
    double dens(double y) const { return alpha * std::sinh(alpha * (R - y)) / cm1; }
    double cdf(double y) const { return 1.0 - (std::cosh(alpha * (R - y)) - 1.0) / cm1; }
};

double share_below(double r1, double r2, double t, double cosh_t) {
    if (t >= r1 + r2) return 1.0;
    if (t <= std::fabs(r1 - r2)) return 0.0;
    const double s = (cosh_t - std::cosh(r1 - r2)) / (2.0 * std::sinh(r1) * std::sinh(r2));
    if (!(s > 0.0)) return 0.0;
    if (s >= 1.0) return 1.0;
    return (2.0 / kPi) * std::asin(std::sqrt(s));
}

double dist_cdf(const Disk& D, double t) {
    const double R = D.R;
    if (t <= 0.0) return 0.0;
    if (t >= 2.0 * R) return 1.0;
    const double ct = std::cosh(t);
    std::vector<double> cuts = {0.0, R};
    for (double c : {R - t, 2.0 * R - t, t})
        if (c > 0.0 && c < R) cuts.push_back(c);
    std::sort(cuts.begin(), cuts.end());
    double ya[kYPanels * kGL], wa[kYPanels * kGL], yb[kYPanels * kGL], wb[kYPanels * kGL];
    double sum = 0.0;
    for (size_t q = 0; q + 1 < cuts.size(); ++q) {
        if (!(cuts[q + 1] > cuts[q])) continue;
        const int na = cos_mapped_rule(cuts[q], cuts[q + 1], kYPanels, ya, wa);
        for (int a = 0; a < na; ++a) {
            const double y1 = ya[a];
            const double lo = std::max(0.0, y1 - t), hi = std::min(R, y1 + t);
            const double full = 2.0 * R - t - y1;  // share = 1 for y2 >= full
            if (!(hi > lo)) continue;
            double in = 0.0;
            if (full <= lo) {
                in = D.cdf(hi) - D.cdf(lo);
            } else {
                const double top = std::min(hi, full);
                const int nb = cos_mapped_rule(lo, top, kYPanels, yb, wb);
                for (int b = 0; b < nb; ++b)
                    in += wb[b] * D.dens(yb[b]) * share_below(R - y1, R - yb[b], t, ct);
                if (full < hi) in += D.cdf(hi) - D.cdf(full);
            }
            sum += wa[a] * D.dens(y1) * in;
        }
    }
    return sum;
}

}  // namespace

void hrg_t_rule(double R, double T, std::vector<double>& ts, std::vector<double>& ws,
                double* tail) {
    // t panels growing geometrically away from R; the logistic weight outside
    // R +- 80 T is below e^-40
    const double s = 2.0 * T, tlo = std::max(0.0, R - 40.0 * s), thi = std::min(2.0 * R, R + 40.0 * s);
    std::vector<double> cuts = {R};
    for (double x = R, w = s; x > tlo; w *= 2.0) cuts.push_back(x = std::max(tlo, x - w));
    for (double x = R, w = s; x < thi; w *= 2.0) cuts.push_back(x = std::min(thi, x + w));
    std::sort(cuts.begin(), cuts.end());
    ts.clear();
    ws.clear();
    double tb[kTPanels * kGL], wtb[kTPanels * kGL];
    for (size_t q = 0; q + 1 < cuts.size(); ++q) {
        if (!(cuts[q + 1] > cuts[q])) continue;
        const int k = cos_mapped_rule(cuts[q], cuts[q + 1], kTPanels, tb, wtb);
        for (int a = 0; a < k; ++a) {
            const double e = std::exp(-std::fabs(tb[a] - R) / s);
            ts.push_back(tb[a]);
            ws.push_back(wtb[a] * e / (s * (1.0 + e) * (1.0 + e)));
        }
    }
    const double eh = std::exp(-(thi - R) / s);
    *tail = eh / (1.0 + eh);  // t beyond thi: the distance CDF is 1 (or the weight negligible)
}

void hrg_unit_y_rule(double* c, double* w) {
    static_assert(kHrgYNodes == kYPanels * kGL, "y rule size");
    cos_mapped_rule(0.0, 1.0, kYPanels, c, w);
}

double hrg_expected_degree(int64_t n, double alpha, double T, double R) {
    const Disk D{alpha, R, std::cosh(alpha * R) - 1.0};
    if (T == 0.0) return (double)(n - 1) * dist_cdf(D, R);
    std::vector<double> ts, ws;
    double tail = 0.0;
    hrg_t_rule(R, T, ts, ws, &tail);
    // the distance CDF at every node, spread over host threads; summed in node order
    std::vector<double> g(ts.size(), 0.0);
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t nthreads = std::min<size_t>(hw, ts.size());
    auto run = [&](size_t th) {
        for (size_t i = th; i < ts.size(); i += nthreads) g[i] = dist_cdf(D, ts[i]);
    };
    std::vector<std::thread> pool;
    std::vector<size_t> mine;  // shares of threads that could not start: this thread's
    for (size_t th = 0; th < nthreads; ++th) {
        try {
            pool.emplace_back(run, th);
        } catch (const std::system_error&) {
            mine.push_back(th);
        }
    }
    for (size_t th : mine) run(th);
    for (auto& t : pool) t.join();
    double p = 0.0;
    for (size_t i = 0; i < ts.size(); ++i) p += ws[i] * g[i];
    p += tail;
    return (double)(n - 1) * p;
}

double hrg_radius_for_degree(int64_t n, double alpha, double T, double target) {
    return hrg_radius_for_degree(n, alpha, T, target,
                                 [&](double R) { return hrg_expected_degree(n, alpha, T, R); });
}

double hrg_radius_for_degree(int64_t n, double alpha, double T, double target,
                             const std::function<double(double)>& E) {
    // start from the large-R limit E ~ K n e^(-R/2), K = 8 alpha^2 / (pi (2 alpha - 1)^2)
    // times pi T / sin(pi T); ln E is nearly linear in R, so the secant method (and as a
    // fallback regula falsi, Illinois) on ln E(R) - ln target converges in a few steps
    double K = 8.0 * alpha * alpha / (kPi * (2.0 * alpha - 1.0) * (2.0 * alpha - 1.0));
    if (T > 0.0) K *= kPi * T / std::sin(kPi * T);
    double r0 = 2.0 * std::log(K * (double)n / target);
    if (!(r0 > 1e-3 && r0 < 700.0)) r0 = std::min(700.0, std::max(1.0, 2.0 * std::log((double)n)));
    auto F = [&](double R) { return std::log(E(R)) - std::log(target); };
    const double f_start = F(r0);
    if (f_start == 0.0) return r0;
    // secant steps from r0 and the point the slope -1/2 of ln E predicts (three to five
    // evaluations to 1e-13); a step that leaves (1e-3, 700) or stalls falls back to the
    // bracketing search below, which starts again from r0
    {
        double a = r0, fa = f_start, b = r0 + 2.0 * f_start;
        if (b > 1e-3 && b < 700.0) {
            double fb = F(b);
            for (int it = 0; it < 30 && std::isfinite(fb); ++it) {
                if (std::fabs(fb) <= 1e-14) return b;
                if (fb == fa) break;
                double c = b - fb * (b - a) / (fb - fa);
                c = std::min(b + 4.0, std::max(b - 4.0, c));
                if (!(c > 1e-3 && c < 700.0)) break;
                if (std::fabs(c - b) <= 1e-13 * b) return c;
                a = b;
                fa = fb;
                b = c;
                fb = F(b);
            }
        }
    }
    double lo = r0, hi = r0, flo = f_start, fhi = flo;
    // F decreases in R: find lo with F >= 0 and hi with F < 0
    for (double step = 0.5; flo < 0.0; step *= 2.0) {
        hi = lo;
        fhi = flo;
        lo = std::max(1e-3, lo - step);
        flo = F(lo);
        if (lo <= 1e-3 && flo < 0.0) return std::nan("");
    }
    for (double step = 0.5; fhi >= 0.0; step *= 2.0) {
        lo = hi;
        flo = fhi;
        hi = std::min(700.0, hi + step);
        fhi = F(hi);
        if (hi >= 700.0 && fhi >= 0.0) return std::nan("");
    }
    int side = 0;
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
        double mid = (it % 6 == 5) ? 0.5 * (lo + hi) : hi - fhi * (hi - lo) / (fhi - flo);
        if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
        const double fm = F(mid);
        if (std::fabs(fm) <= 1e-14) return mid;
        if (fm >= 0.0) {
            lo = mid;
            flo = fm;
            if (side == 1) fhi *= 0.5;
            side = 1;
        } else {
            hi = mid;
            fhi = fm;
            if (side == -1) flo *= 0.5;
            side = -1;
        }
    }
    return 0.5 * (lo + hi);
}

}  // namespace gg
