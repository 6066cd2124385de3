// Host-side 1D ingredients of the spectral finite-element basis (Sec. 2.3, Eq. fem):
// Gauss-Lobatto-Legendre nodes/weights (the quadrature that makes M diagonal, text
// after Eq. hep), Gauss-Legendre rules for the local-potential term (Eq. quadLocal),
// and Lagrange tables in barycentric form (Berrut & Trefethen, SIAM Rev. 2004).
#include "internal.h"

#include <cmath>

namespace dftfe {

namespace {
// P_n(x) and P_{n-1}(x) by the three-term recurrence (n >= 1).
void legendre_pair(int n, double x, double* pn, double* pnm1) {
  double p0 = 1.0, p1 = x;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

void symmetrise(std::vector<double>& x, std::vector<double>& w) {
  const int n = (int)x.size();
  for (int i = 0; i < n / 2; ++i) {
    double xs = 0.5 * (x[n - 1 - i] - x[i]);
    double ws = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = -xs;
    x[n - 1 - i] = xs;
    w[i] = w[n - 1 - i] = ws;
  }
  if (n % 2) x[n / 2] = 0.0;
}
}  // namespace

Rule1D gll_rule(int p) {
  Rule1D r;
  r.x.assign(p + 1, 0.0);
  r.w.assign(p + 1, 0.0);
  r.x[0] = -1.0;
  r.x[p] = 1.0;
  // interior nodes: roots of P_p'(x); Newton with P_p'' from Legendre's equation
  for (int i = 1; i < p; ++i) {
    double x = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre_pair(p, x, &pn, &pm);
      double d1 = p * (x * pn - pm) / (x * x - 1.0);
      double d2 = (2.0 * x * d1 - p * (p + 1.0) * pn) / (1.0 - x * x);
      double dx = d1 / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    r.x[i] = x;
  }
  for (int i = 0; i <= p; ++i) {
    double pn, pm;
    legendre_pair(p, r.x[i], &pn, &pm);
    r.w[i] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
  symmetrise(r.x, r.w);
  return r;
}

Rule1D gauss_rule(int n) {
  Rule1D r;
  r.x.assign(n, 0.0);
  r.w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double d1 = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre_pair(n, x, &pn, &pm);
      if (n == 1) pm = 1.0;
      d1 = n * (x * pn - pm) / (x * x - 1.0);
      double dx = pn / d1;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double pn, pm;
    legendre_pair(n, x, &pn, &pm);
    if (n == 1) pm = 1.0;
    d1 = n * (x * pn - pm) / (x * x - 1.0);
    r.x[i] = x;
    r.w[i] = 2.0 / ((1.0 - x * x) * d1 * d1);
  }
  symmetrise(r.x, r.w);
  return r;
}

std::vector<double> barycentric_weights(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (x[j] - x[m]);
  return lam;
}

std::vector<double> lagrange_at(const std::vector<double>& x, const std::vector<double>& pts) {
  const int n = (int)x.size();
  const auto lam = barycentric_weights(x);
  std::vector<double> T(pts.size() * n, 0.0);
  for (size_t q = 0; q < pts.size(); ++q) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (pts[q] == x[j]) hit = j;
    if (hit >= 0) {
      T[q * n + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += lam[j] / (pts[q] - x[j]);
    for (int j = 0; j < n; ++j) T[q * n + j] = (lam[j] / (pts[q] - x[j])) / den;
  }
  return T;
}

std::vector<double> derivative_matrix(const std::vector<double>& x) {
  const int n = (int)x.size();
  const auto lam = barycentric_weights(x);
  std::vector<double> D(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * n + j] = v;
      diag -= v;
    }
    D[i * n + i] = diag;
  }
  return D;
}

}  // namespace dftfe
