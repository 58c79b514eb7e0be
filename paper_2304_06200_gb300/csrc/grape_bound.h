// Host-side error bound E_A(m, s) and (m, s) rule (Sec. III.B, App. C).
#pragma once

#include <vector>

namespace grape {

double unit_roundoff(int precision);
double tail_remainder(double b, int m);
double error_bound(double x, int m, int s, int sigma, double u);
bool select_ms(double x, double tau, int sigma, double u, int m_max, int s_max, int* m_out, int* s_out);

// Breakpoint table: X[(s-1)*m_cap + (m-1)] = largest ||A||_1 with E_A(m, s) <= tau (-1 if none),
// smax[s-1] = max_m X.  Rows are added until smax reaches x_enough or the feasible range has
// clearly peaked (rounding dominates) or s_limit rows exist.
struct ScheduleTable {
  int m_cap = 0, s_cap = 0;
  double x_max = -1.0;
  std::vector<double> X;
  std::vector<double> smax;
};

ScheduleTable build_table(double tau, int sigma, double u, int m_max, int s_limit, double x_enough, int s_min_rows = 1);
bool table_lookup(const ScheduleTable& t, double x, int* m_out, int* s_out);

}  // namespace grape
