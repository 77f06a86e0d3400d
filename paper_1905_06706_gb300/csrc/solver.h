// Expected average degree f(c) and the search for c (Sec. 4.1, App. B.2).
#pragma once
#include <stdint.h>

#include <cmath>
#include <functional>
#include <vector>

namespace gg {

// Expected average degree f(K) of a GIRG with given weights (App. B.2) as a function
// of the model's scale K (c^T, or c^d at T = 0; Eq. 1 reads p = min{1, (K q/r^d)^(1/T)}).
// For a pair with z = 2^d K w_u w_v / W, E[X_uv] = 1 when z >= 1 (the pairs E_R) and
// (z - T z^(1/T)) / (1 - T) otherwise.  The weights are split at a threshold thr: the
// "top" weights above it are held sorted, the rest only through four sums.  While no
// rest weight can be in an E_R pair (2^d K thr w_max / W < 1), f needs per-vertex work
// only over the top weights; every power w^(1/T) is formed as (w / thr)^(1/T) <= 1 or
// inside a log-sum-exp, so small T neither overflows nor cancels.
class DegreeModel {
   public:
    DegreeModel(int64_t n, int d, double T, double W) : n_(n), d_(d), T_(T), W_(W) {}
    // top: every weight above thr, in decreasing order; rest sums over weights <= thr:
    // sw = sum w, s2 = sum w^2, sx = sum (w/thr)^(1/T), sx2 = sum (w/thr)^(2/T).
    void set_split(double thr, std::vector<double> top, double sw, double s2, double sx,
                   double sx2);
    // the split stays exact for this K (no rest weight in an E_R pair)
    bool valid(double K) const;
    // the largest threshold that is valid at K
    double needed_threshold(double K) const;
    // f(K); with slope, also K f'(K)
    double f(double K, double* slope = nullptr) const;
    // K with f(K) = target; fetch(t) must call set_split with a threshold <= t
    double solve(double target, const std::function<void(double)>& fetch);

   private:
    int64_t n_;
    int d_;
    double T_, W_;
    double thr_ = 0.0, sw_ = 0.0, s2_ = 0.0, sx_ = 0.0, sx2_ = 0.0;
    // over the top weights (decreasing), all independent of K: b = log(w)/T, suffix
    // sums of w and w^2, and the suffix sums of w^(1/T) and w^(2/T) scaled by the
    // suffix's first term: sum_{j >= k} e_j = exp(b_k) sr_[k], sum e_j^2 = exp(2 b_k)
    // sr2_[k], e = w^(1/T) (no power of a weight is formed, whatever T)
    std::vector<double> top_, b_, suf_, suf2_, sr_, sr2_;
    // when 1/T is an integer mi <= 8: y = (w/thr)^mi (>= 1, no overflow) and suffix sums
    // of y and y^2, so that z^(1/T) = (A thr^2)^mi y_u y_v needs no exp
    int mi_ = 0;
    std::vector<double> py_, spy_, spy2_;
};

}  // namespace gg

namespace gg {

// Expected average degree of an HRG with n vertices, dispersion alpha, temperature T
// and disk radius R (Sec. 2.2), and the R that gives a target degree.  The paper
// gives no formula; this integrates the model's definition: (n - 1) times the
// probability that two random vertices are adjacent, which is P(dist < R) at T = 0
// and E[P(dist < t)] over t ~ logistic(R, 2T) at T > 0.
double hrg_expected_degree(int64_t n, double alpha, double T, double R);
// R with hrg_expected_degree(n, alpha, T, R) = target (NaN if none in (0, 700)).
double hrg_radius_for_degree(int64_t n, double alpha, double T, double target);
// The same search with another evaluation of the expected degree E(R).
double hrg_radius_for_degree(int64_t n, double alpha, double T, double target,
                             const std::function<double(double)>& E);

// The pieces of the T > 0 quadrature, for evaluating it elsewhere (the device):
// t nodes and weights (with the logistic density folded in) so that
// P(adjacent) = sum_i ws[i] P(dist < ts[i]) + *tail;
void hrg_t_rule(double R, double T, std::vector<double>& ts, std::vector<double>& ws,
                double* tail);
// and the y rule on [0, 1] that P(dist < t) applies to each of its intervals [a, b]
// (nodes a + (b - a) c[k], weights (b - a) w[k], k < kHrgYNodes).
constexpr int kHrgYNodes = 30;
void hrg_unit_y_rule(double* c, double* w);

}  // namespace gg
