// Host-side reference data: Gauss rules, 1D Lagrange tables, element sizes.
//
// Gauss-Legendre points are the roots of P_n, found by Newton's method from
// the Chebyshev-like first guess cos(pi (i + 3/4) / (n + 1/2)); weights
// 2 / ((1 - x^2) P_n'(x)^2).  Gauss-Lobatto points are +-1 and the roots of
// P_{n-1}', Newton on P_{n-1}' with P_{n-1}'' from Legendre's equation
// (1 - x^2) P'' = 2 x P' - N (N + 1) P.  Everything is mapped to [0, 1].
#include <algorithm>
#include <cmath>

#include "dpg_internal.h"

namespace dpg {

static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *P = p1;
  // P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), valid in the open interval
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre01(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, &P, &dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, &P, &dP);
    x[i] = 0.5 * (z + 1.0);
    w[i] = 1.0 / ((1.0 - z * z) * dP * dP);  // (2 / ((1-z^2) P'^2)) / 2
  }
  // ascending order
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (x[j] < x[i]) {
        std::swap(x[i], x[j]);
        std::swap(w[i], w[j]);
      }
}

void gauss_lobatto01(int n, double* x) {
  const double pi = 3.14159265358979323846;
  const int N = n - 1;
  x[0] = 0.0;
  x[n - 1] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(pi * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(N, z, &P, &dP);
      double d2P = (2.0 * z * dP - N * (N + 1.0) * P) / (1.0 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (z + 1.0);
  }
  std::sort(x, x + n);
}

void lagrange1d(const double* z, int n, double x, double* val, double* der) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (x - z[m]) / (z[j] - z[m]);
    val[j] = v;
    double d = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == j) continue;
      double t = 1.0 / (z[j] - z[k]);
      for (int m = 0; m < n; ++m)
        if (m != j && m != k) t *= (x - z[m]) / (z[j] - z[m]);
      d += t;
    }
    der[j] = d;
  }
}

Sizes make_sizes(int p) {
  Sizes s{};
  s.p = p;
  s.r = p + 1;
  s.rt = p + 2;
  s.nq1 = p + 3;
  s.nq = s.nq1 * s.nq1 * s.nq1;
  s.nqf = s.nq1 * s.nq1;
  s.n_f = 3 * s.rt * (s.rt + 1) * (s.rt + 1);
  s.n_v = 2 * s.n_f;
  s.nL = (p + 1) * (p + 1) * (p + 1);
  s.n_u = 6 * s.nL;
  s.nt = 12 * s.r * s.r;
  s.n_h = 2 * s.nt;
  s.N = s.n_v + s.n_u + s.n_h + 1;
  return s;
}

void build_tables(int p, Tables* t) {
  *t = Tables{};
  t->p = p;
  t->r = p + 1;
  t->rt = p + 2;
  t->nq1 = p + 3;
  t->npt = t->nq1 + 2;
  gauss_legendre01(t->nq1, t->pt, t->w);
  t->pt[t->nq1] = 0.0;
  t->pt[t->nq1 + 1] = 1.0;
  double nodes[NFAM][MAXF1D], dummy[MAXF1D];
  t->nfun[F_OPEN_T] = t->rt;
  gauss_legendre01(t->rt, nodes[F_OPEN_T], dummy);
  t->nfun[F_CLOSED_T] = t->rt + 1;
  gauss_lobatto01(t->rt + 1, nodes[F_CLOSED_T]);
  t->nfun[F_OPEN_R] = t->r;
  gauss_legendre01(t->r, nodes[F_OPEN_R], dummy);
  t->nfun[F_CLOSED_R] = t->r + 1;
  gauss_lobatto01(t->r + 1, nodes[F_CLOSED_R]);
  t->nfun[F_L2] = p + 1;
  gauss_legendre01(p + 1, nodes[F_L2], dummy);
  for (int f = 0; f < NFAM; ++f)
    for (int q = 0; q < t->npt; ++q)
      lagrange1d(nodes[f], t->nfun[f], t->pt[q], t->val[f][q], t->der[f][q]);
}

std::vector<int> trace_functions(int r) {
  std::vector<int> out;
  for (int c = 0; c < 3; ++c) {
    int n[3] = {r + 1, r + 1, r + 1};
    n[c] = r;
    for (int i2 = 0; i2 < n[2]; ++i2)
      for (int i1 = 0; i1 < n[1]; ++i1)
        for (int i0 = 0; i0 < n[0]; ++i0) {
          int ii[3] = {i0, i1, i2};
          bool tr = false;
          for (int d = 0; d < 3; ++d)
            if (d != c && (ii[d] == 0 || ii[d] == r)) tr = true;
          if (tr) out.push_back(pack_fun(c, i0, i1, i2));
        }
  }
  return out;
}

}  // namespace dpg
