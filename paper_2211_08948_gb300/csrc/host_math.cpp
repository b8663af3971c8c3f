// Host-side float64 scalar math of the Leja method (Sec. 2.2):
//   phi_l(z) for real z (Sec. 1), the real Leja sequence on [-2, 2], and
//   Newton divided differences.  O(m^2) work per table, done once per pass.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "phix_internal.h"

namespace phix {

// phi_l(z) = sum_k z^k / (k+l)!  for |z| < l + 1 (where the recurrence
// cancels), else phi_0 = e^z and phi_{j+1} = (phi_j - 1/j!) / z.
double phi_host(int l, double z) {
  if (l == 0) return std::exp(z);
  if (std::fabs(z) < l + 1.0) {
    double inv_fact = 1.0;
    for (int j = 2; j <= l; ++j) inv_fact /= j;
    double term = inv_fact, sum = 0.0;
    for (int k = 0; k < 80; ++k) {
      sum += term;
      term *= z / (k + l + 1);
      if (std::fabs(term) < 1e-18 * std::fabs(sum)) {
        sum += term;
        break;
      }
    }
    return sum;
  }
  double p = std::exp(z);
  double inv_fact = 1.0;  // 1/j!
  for (int j = 0; j < l; ++j) {
    p = (p - inv_fact) / z;
    inv_fact /= (j + 1);
  }
  return p;
}

// The next Leja point: for every gap between consecutive existing points
// the unique zero of L'(x) = sum 1/(x - xi_i) (L = log prod|x - xi_i|) is
// located by a safeguarded Newton iteration; the gap with the largest L
// wins, exact ties going to the smaller x.
static double next_leja(const std::vector<double>& pts) {
  std::vector<double> s(pts);
  std::sort(s.begin(), s.end());
  double best_x = 0.0, best_L = -INFINITY;
  const size_t n = pts.size();
  for (size_t g = 0; g + 1 < s.size(); ++g) {
    double lo = s[g], hi = s[g + 1];
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
      double f = 0.0, df = 0.0;
      for (size_t i = 0; i < n; ++i) {
        double r = 1.0 / (x - pts[i]);
        f += r;
        df -= r * r;
      }
      if (f > 0.0)
        lo = x;
      else
        hi = x;
      double xn = x - f / df;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      double step = std::fabs(xn - x);
      x = xn;
      if (step <= 2.0 * std::nextafter(std::fabs(x), INFINITY) - 2.0 * std::fabs(x)) break;
    }
    double L = 0.0;
    for (size_t i = 0; i < n; ++i) L += std::log(std::fabs(x - pts[i]));
    const double thr = 1e-12 * std::fmax(1.0, std::fabs(best_L));
    if (L > best_L + thr) {
      best_L = L;
      best_x = x;
    } else if (L >= best_L - thr && x < best_x) {
      best_x = x;
      if (L > best_L) best_L = L;
    }
  }
  return best_x;
}

int leja_points_host(double* xi, int m) {
  if (m < 1 || m > 4096) return 1;
  const double* t = leja_table(m);
  std::memcpy(xi, t, sizeof(double) * m);
  return 0;
}

const double* leja_table(int m) {
  static std::mutex mu;
  static std::vector<double> table;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)table.size() < m) {
    if (table.empty()) {
      table.reserve(4096);  // returned pointers stay valid as the table grows
      table.push_back(2.0);
      if (m > 1) table.push_back(-2.0);
      if (m > 2) table.push_back(0.0);
    }
    while ((int)table.size() < m) table.push_back(next_leja(table));
  }
  return table.data();
}

// d_j = f[x_0, ..., x_j] in place (standard recursion).
void divided_differences_host(const double* x, double* f, int n) {
  for (int j = 1; j < n; ++j)
    for (int i = n - 1; i >= j; --i) f[i] = (f[i] - f[i - 1]) / (x[i] - x[i - j]);
}

void DDTable::grow(int n) {
  const int n0 = (int)d.size();
  if (n0 >= n) return;
  const double* x = leja_table(n);
  // The new points i = n0 .. n-1 column by column: column j holds
  // f[x_{i-j}, ..., x_i] = (f[x_{i-j+1}..x_i] - f[x_{i-j}..x_{i-1}]) / (x_i - x_{i-j}),
  // the entry at i = n0 taking its left neighbour from the stored diagonal of
  // point n0 - 1.  The same operations as point-by-point growth, in an order
  // whose inner loop has independent divisions.
  const int C = n - n0;
  std::vector<double> col(C), nxt(C), ndiag(n);
  for (int c = 0; c < C; ++c) col[c] = phi_host(l, a + b * x[n0 + c]);
  d.resize(n);
  if (n0 == 0) d[0] = col[0];
  ndiag[0] = col[C - 1];
  for (int j = 1; j < n; ++j) {
    const int c0 = std::max(0, j - n0);
    const double* __restrict__ cv = col.data();
    double* __restrict__ nv = nxt.data();
    const double* __restrict__ xi = x + n0;
    int c = c0;
    if (c == 0) {
      nv[0] = (cv[0] - diag[j - 1]) / (xi[0] - xi[-j]);
      c = 1;
    }
    for (; c < C; ++c) nv[c] = (cv[c] - cv[c - 1]) / (xi[c] - xi[c - j]);
    col.swap(nxt);
    if (j >= n0) d[j] = col[j - n0];
    ndiag[j] = col[C - 1];
  }
  diag.swap(ndiag);
}

}  // namespace phix
