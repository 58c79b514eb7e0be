// The (m, s) rule of Sec. III.B with the error bound E_A(m, s) of App. C, on the host.
//
//   x = ||A||_1 (A = -i H dt), b = x / s, u = unit roundoff, sigma = sigma' (Eq. (sigmapdef)).
//   R_m(b)  = sum_{q > m} b^q / q!                                      (App. C.1)
//   eps_t  <= s R (1 - (s R)^s) / (1 - s R),  requires s R < 1           (Eq. (truncation))
//   u'      = 2 sqrt(2) u / (1 - 2u),  gamma_n = n u' / (1 - n u')        (App. C.2)
//   beta    = sum_{k=0}^m gamma_{k(sigma+2)+m+2} b^k / k!                  (Eq. (B23))
//   alpha   = 1 + R_m(b)
//   eps_r  <= (alpha + beta)^s - alpha^s                                  (Eq. (rouding))
//   E_A     = eps_t bound + eps_r bound                                    (Eq. (overallupperbound))
// Rule: the smallest s for which some m <= m_max has E_A <= tau, then the smallest such m.
//
// For the device, E_A is tabulated as breakpoints: E_A is increasing in x for fixed (m, s),
// so X[s][m] = sup { x : E_A(x; m, s) <= tau } turns the rule into comparisons.
#include "grape_bound.h"

#include <cmath>
#include <limits>
#include <vector>

namespace grape {

double unit_roundoff(int precision) { return precision == 1 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53); }

static double gamma_n(double n, double up) {
  const double nu = n * up;
  if (nu >= 1.0) return std::numeric_limits<double>::infinity();
  return nu / (1.0 - nu);
}

// R_m(b) by a forward tail sum starting at q = m + 1 (no e^b - partial-sum cancellation).
double tail_remainder(double b, int m) {
  if (!(b > 0.0)) return 0.0;
  const double logt = (m + 1) * std::log(b) - std::lgamma(m + 2.0);
  if (logt > 700.0) return std::numeric_limits<double>::infinity();
  double term = std::exp(logt), total = 0.0;
  for (int q = m + 1;; ) {
    total += term;
    ++q;
    term *= b / q;
    if (q > b && term <= total * 1e-18) break;
    if (total > 1e300) return std::numeric_limits<double>::infinity();
  }
  return total;
}

double error_bound(double x, int m, int s, int sigma, double u) {
  if (m < 1 || s < 1 || !(x >= 0.0)) return std::numeric_limits<double>::infinity();
  const double b = x / s;
  const double R = tail_remainder(b, m);
  const double sR = s * R;
  if (!(sR < 1.0)) return std::numeric_limits<double>::infinity();
  const double trunc = sR * (1.0 - std::pow(sR, s)) / (1.0 - sR);
  const double up = 2.0 * std::sqrt(2.0) * u / (1.0 - 2.0 * u);
  double beta = 0.0, bk = 1.0;   // bk = b^k / k!
  for (int k = 0; k <= m; ++k) {
    if (k > 0) bk *= b / k;
    beta += gamma_n(double(k) * (sigma + 2) + m + 2, up) * bk;
  }
  const double alpha = 1.0 + R;
  // (alpha + beta)^s - alpha^s = alpha^s * expm1(s * log1p(beta / alpha)), free of cancellation.
  const double eps_r = std::pow(alpha, s) * std::expm1(s * std::log1p(beta / alpha));
  return trunc + eps_r;
}

bool select_ms(double x, double tau, int sigma, double u, int m_max, int s_max, int* m_out, int* s_out) {
  for (int s = 1; s <= s_max; ++s)
    for (int m = 1; m <= m_max; ++m)
      if (error_bound(x, m, s, sigma, u) <= tau) { *m_out = m; *s_out = s; return true; }
  return false;
}

// Largest x with E_A(x; m, s) <= tau (E_A increases with x), or -1 if even x = 0 fails.
static double breakpoint(int m, int s, int sigma, double u, double tau) {
  if (!(error_bound(0.0, m, s, sigma, u) <= tau)) return -1.0;
  double lo = 0.0, hi = 1.0;
  while (error_bound(hi, m, s, sigma, u) <= tau) {
    lo = hi;
    hi *= 2.0;
    if (hi > 1e6) return lo;
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (error_bound(mid, m, s, sigma, u) <= tau) lo = mid; else hi = mid;
  }
  return lo;
}

ScheduleTable build_table(double tau, int sigma, double u, int m_max, int s_limit, double x_enough, int s_min_rows) {
  ScheduleTable t;
  t.m_cap = m_max;
  double best = -1.0;
  int best_s = 0, since_best = 0;
  for (int s = 1; s <= s_limit; ++s) {
    double smax = -1.0;
    std::vector<double> row(m_max, -1.0);
    for (int m = 1; m <= m_max; ++m) {
      row[m - 1] = breakpoint(m, s, sigma, u, tau);
      smax = std::max(smax, row[m - 1]);
    }
    t.X.insert(t.X.end(), row.begin(), row.end());
    t.smax.push_back(smax);
    t.s_cap = s;
    if (smax > best) { best = smax; best_s = s; since_best = 0; } else { ++since_best; }
    if (s < s_min_rows) continue;
    if (best >= x_enough) break;
    // Past the peak, rounding dominates and larger s only shrinks the feasible range.
    if (best_s > 0 && since_best >= 16 && s >= 2 * best_s) break;
  }
  t.x_max = best;
  return t;
}

bool table_lookup(const ScheduleTable& t, double x, int* m_out, int* s_out) {
  for (int s = 1; s <= t.s_cap; ++s) {
    if (t.smax[s - 1] >= x) {
      for (int m = 1; m <= t.m_cap; ++m)
        if (t.X[(s - 1) * t.m_cap + (m - 1)] >= x) { *m_out = m; *s_out = s; return true; }
    }
  }
  return false;
}

}  // namespace grape
