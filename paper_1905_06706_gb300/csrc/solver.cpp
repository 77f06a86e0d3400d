// Expected average degree of a GIRG and the search for c (Sec. 4.1, App. B.2).
//
// f(c) = E[average degree] = (1/n) sum over ordered pairs u != v of E[X_uv].
// Without the min of Eq. 1, E[X_uv] has the closed form
//   T > 0:  c^T 2^d/(1-T) q - c 2^(d/T)/(1/T - 1) q^(1/T),   q = w_u w_v / W
//   T = 0:  2^d c^d q
// whose double sums reduce to sums of w, w^2, w^(1/T), w^(2/T).  Pairs where the
// min takes effect (the set E_R: c^T q > 2^-d, resp. 2^d c^d q > 1) have
// E[X_uv] = 1; their error is subtracted by walking the heaviest vertices in
// decreasing weight, where each vertex's partners form a prefix (App. B.2).
// The search brackets c by doubling / halving and bisects on log c.
#include "solver.h"

#include <algorithm>
#include <cmath>
#include <thread>

namespace gg {

DegreeModel::DegreeModel(int64_t n, int d, double T, double W, double s2, double st, double s2t)
    : n_(n), d_(d), T_(T), W_(W) {
    S1_ = W - s2 / W;
    S2_ = T > 0.0 ? (st * st - s2t) / std::pow(W, 1.0 / T) : 0.0;
    wmax_ = 0.0;
    have_thr_ = INFINITY;
}

void DegreeModel::set_top(std::vector<double> top, double fetched_above, bool descending) {
    if (!descending) std::sort(top.begin(), top.end(), [](double a, double b) { return a > b; });
    top_ = std::move(top);
    have_thr_ = fetched_above;
    if (!top_.empty()) wmax_ = std::max(wmax_, top_[0]);
    pre_w_.assign(top_.size() + 1, 0.0);
    pre_wt_.assign(top_.size() + 1, 0.0);
    wt_.assign(top_.size(), 0.0);
    for (size_t a = 0; a < top_.size(); ++a) {
        wt_[a] = T_ > 0.0 ? power(top_[a]) : 0.0;
        pre_w_[a + 1] = pre_w_[a] + top_[a];
        pre_wt_[a + 1] = pre_wt_[a] + wt_[a];
    }
    WT_ = T_ > 0.0 ? power(W_) : 1.0;
}

// x^(1/T): repeated products when 1/T is a small integer.
double DegreeModel::power(double x) const {
    const double e = 1.0 / T_;
    if (e == std::floor(e) && e <= 16.0) {
        double r = x;
        for (int q = 1; q < (int)e; ++q) r *= x;
        return r;
    }
    return std::pow(x, e);
}

double DegreeModel::qstar(double c) const {
    if (T_ == 0.0) return 1.0 / std::ldexp(std::pow(c, d_), d_);
    return std::ldexp(1.0, -d_) / std::pow(c, T_);
}

double DegreeModel::needed_threshold(double c) const {
    // both endpoints of a pair in E_R weigh more than qstar W / w_max
    return qstar(c) * W_ / wmax_;
}

double DegreeModel::f(double c) const {
    const int d = d_;
    const double T = T_;
    double main_term;
    double a1 = 0.0, a2 = 0.0;
    if (T == 0.0) {
        a1 = std::ldexp(std::pow(c, d), d);
        main_term = a1 * S1_;
    } else {
        a1 = std::pow(c, T) * std::ldexp(1.0, d) / (1.0 - T);
        a2 = c * std::pow(2.0, d / T) / (1.0 / T - 1.0);
        main_term = a1 * S1_ - a2 * S2_;
    }
    const double qs = qstar(c);
    double err = 0.0;
    // partners of the heaviest vertex: the prefix of weights above qs W / w_max
    // (binary search); for lighter vertices the prefix only shrinks
    size_t k = 0;
    if (!top_.empty()) {
        const double lim0 = qs * W_ / top_[0];
        k = (size_t)(std::upper_bound(top_.begin(), top_.end(), lim0,
                                      [](double x, double y) { return x > y; }) -
                     top_.begin());
    }
    for (size_t a = 0; a < top_.size(); ++a) {
        const double wu = top_[a];
        const double lim = qs * W_ / wu;
        while (k > 0 && !(top_[k - 1] > lim)) --k;
        if (k == 0) break;
        double cnt = (double)k, sw = pre_w_[k], swt = pre_wt_[k];
        if (a < k) {
            cnt -= 1.0;
            sw -= wu;
            if (T > 0.0) swt -= wt_[a];
        }
        if (cnt <= 0.0) continue;
        double s;
        if (T == 0.0)
            s = a1 * (wu / W_) * sw;
        else
            s = a1 * (wu / W_) * sw - a2 * (wt_[a] / WT_) * swt;
        err += s - cnt;
    }
    return (main_term - err) / (double)n_;
}

double DegreeModel::solve(double target, const std::function<void(double)>& fetch) {
    auto eval = [&](double c) {
        const double need = needed_threshold(c);
        if (need < have_thr_) fetch(0.5 * need);
        return f(c);
    };
    // start from the c at which the leading term of f alone reaches the target
    // (c^T 2^d S1 / ((1 - T) n) = target, or 2^d c^d S1 / n = target at T = 0);
    // the other terms only lower f, so the root lies near or above it
    double c0;
    if (T_ == 0.0)
        c0 = std::pow(target * (double)n_ / (std::ldexp(1.0, d_) * S1_), 1.0 / d_);
    else
        c0 = std::pow(target * (double)n_ * (1.0 - T_) / (std::ldexp(1.0, d_) * S1_), 1.0 / T_);
    if (!(c0 > 1e-300 && c0 < 1e300)) c0 = 1.0;
    // bracket with steps growing from 5% (the root is usually within a few percent
    // of c0, and small steps keep the needed weights within those already fetched)
    double lo = c0, hi = c0;
    if (eval(c0) < target) {
        for (double f = 1.05; eval(hi) < target && hi < 1e300; f = f * f) {
            lo = hi;
            hi *= f;
        }
    } else {
        for (double f = 1.05; eval(lo) >= target && lo > 1e-300; f = f * f) {
            hi = lo;
            lo /= f;
        }
    }
    // Illinois variant of regula falsi on log c: the bracket [lo, hi] with
    // f(lo) < target <= f(hi) shrinks superlinearly; bisection steps guard it
    double flo = eval(lo) - target, fhi = eval(hi) - target;
    int side = 0;
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
        double mid;
        const double a = std::log(lo), b = std::log(hi);
        if (it % 8 == 7 || !(fhi > flo)) {
            mid = std::sqrt(lo * hi);
        } else {
            mid = std::exp(b - fhi * (b - a) / (fhi - flo));
        }
        if (!(mid > lo && mid < hi)) mid = std::sqrt(lo * hi);
        if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
        const double fm = eval(mid) - target;
        if (fm < 0.0) {
            lo = mid;
            flo = fm;
            if (side == -1) fhi *= 0.5;
            side = -1;
        } else {
            hi = mid;
            fhi = fm;
            if (side == 1) flo *= 0.5;
            side = 1;
        }
        if (std::fabs(fm) <= 1e-14 * target) return mid;
    }
    return 0.5 * (lo + hi);
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

double hrg_expected_degree(int64_t n, double alpha, double T, double R) {
    const Disk D{alpha, R, std::cosh(alpha * R) - 1.0};
    if (T == 0.0) return (double)(n - 1) * dist_cdf(D, R);
    // t panels growing geometrically away from R; the logistic weight outside
    // R +- 80 T is below e^-40
    const double s = 2.0 * T, tlo = std::max(0.0, R - 40.0 * s), thi = std::min(2.0 * R, R + 40.0 * s);
    std::vector<double> cuts = {R};
    for (double x = R, w = s; x > tlo; w *= 2.0) cuts.push_back(x = std::max(tlo, x - w));
    for (double x = R, w = s; x < thi; w *= 2.0) cuts.push_back(x = std::min(thi, x + w));
    std::sort(cuts.begin(), cuts.end());
    std::vector<double> ts, ws;
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
    // the distance CDF at every node, spread over host threads; summed in node order
    std::vector<double> g(ts.size(), 0.0);
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t nthreads = std::min<size_t>(hw, ts.size());
    std::vector<std::thread> pool;
    for (size_t th = 0; th < nthreads; ++th)
        pool.emplace_back([&, th] {
            for (size_t i = th; i < ts.size(); i += nthreads) g[i] = dist_cdf(D, ts[i]);
        });
    for (auto& t : pool) t.join();
    double p = 0.0;
    for (size_t i = 0; i < ts.size(); ++i) p += ws[i] * g[i];
    const double eh = std::exp(-(thi - R) / s);
    p += eh / (1.0 + eh);  // t beyond thi: the distance CDF is 1 (or the weight negligible)
    return (double)(n - 1) * p;
}

double hrg_radius_for_degree(int64_t n, double alpha, double T, double target) {
    // start from the large-R limit E ~ K n e^(-R/2), K = 8 alpha^2 / (pi (2 alpha - 1)^2)
    // times pi T / sin(pi T); ln E is nearly linear in R, so regula falsi (Illinois)
    // on ln E(R) - ln target converges in a few steps
    double K = 8.0 * alpha * alpha / (kPi * (2.0 * alpha - 1.0) * (2.0 * alpha - 1.0));
    if (T > 0.0) K *= kPi * T / std::sin(kPi * T);
    double r0 = 2.0 * std::log(K * (double)n / target);
    if (!(r0 > 1e-3 && r0 < 700.0)) r0 = std::min(700.0, std::max(1.0, 2.0 * std::log((double)n)));
    auto F = [&](double R) { return std::log(hrg_expected_degree(n, alpha, T, R)) - std::log(target); };
    double lo = r0, hi = r0, flo = F(r0), fhi = flo;
    if (flo == 0.0) return r0;
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
