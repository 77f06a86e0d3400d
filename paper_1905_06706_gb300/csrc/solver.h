// Expected average degree f(c) and the search for c (Sec. 4.1, App. B.2).
#pragma once
#include <stdint.h>

#include <functional>
#include <vector>

namespace gg {

class DegreeModel {
   public:
    // s2 = sum w^2, st = sum w^(1/T), s2t = sum w^(2/T) (T > 0).
    DegreeModel(int64_t n, int d, double T, double W, double s2, double st, double s2t);
    // The heaviest weights: every weight strictly above `fetched_above` (`descending`:
    // already in decreasing order).
    void set_top(std::vector<double> top, double fetched_above, bool descending = false);
    void set_wmax(double wmax) { wmax_ = wmax; }
    double f(double c) const;
    // Weight threshold below which no vertex has a partner in E_R at this c.
    double needed_threshold(double c) const;
    // c with f(c) = target; `fetch(t)` must call set_top with all weights above t.
    double solve(double target, const std::function<void(double)>& fetch);

   private:
    double qstar(double c) const;
    double power(double x) const;
    int64_t n_;
    int d_;
    double T_, W_, S1_, S2_, wmax_, have_thr_, WT_ = 1.0;
    std::vector<double> top_, pre_w_, pre_wt_, wt_;
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

}  // namespace gg
