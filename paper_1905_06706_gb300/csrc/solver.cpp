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

namespace gg {

DegreeModel::DegreeModel(int64_t n, int d, double T, double W, double s2, double st, double s2t)
    : n_(n), d_(d), T_(T), W_(W) {
    S1_ = W - s2 / W;
    S2_ = T > 0.0 ? (st * st - s2t) / std::pow(W, 1.0 / T) : 0.0;
    wmax_ = 0.0;
    have_thr_ = INFINITY;
}

void DegreeModel::set_top(std::vector<double> top, double fetched_above) {
    std::sort(top.begin(), top.end(), [](double a, double b) { return a > b; });
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
    double lo = c0, hi = c0;
    if (eval(c0) < target) {
        while (eval(hi) < target && hi < 1e300) hi *= 2.0;
        lo = hi / 2.0;
    } else {
        while (eval(lo) >= target && lo > 1e-300) lo /= 2.0;
        hi = lo * 2.0;
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
