// Host construction of the 1D FR operators (Sec. 2.2): Gauss-Legendre solution
// points, Lagrange interpolation/differentiation, the DG (left/right Radau)
// correction-function derivatives, Legendre modal transforms, and the mortar
// interpolation / L2 projection between degrees.
#include <cmath>
#include <cstring>

#include "fr_internal.h"

namespace frgb {

double legendre_p(int n, double x) {
  double p0 = 1.0, p1 = x;
  if (n == 0) return p0;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double legendre_dp(int n, double x) {
  // P'_n from P'_{k+1} = P'_{k-1} + (2k+1) P_k
  if (n == 0) return 0.0;
  double d0 = 0.0, d1 = 1.0;
  for (int k = 1; k < n; ++k) {
    double d2 = d0 + (2 * k + 1) * legendre_p(k, x);
    d0 = d1;
    d1 = d2;
  }
  return d1;
}

void gauss_legendre(int P, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < P; ++i) {
    // i-th root counted from +1; Newton from the Chebyshev-like guess
    double r = std::cos(pi * (4.0 * (i + 1) - 1.0) / (4.0 * P + 2.0));
    for (int it = 0; it < 100; ++it) {
      double dr = legendre_p(P, r) / legendre_dp(P, r);
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    double d = legendre_dp(P, r);
    x[P - 1 - i] = r;
    w[P - 1 - i] = 2.0 / ((1.0 - r * r) * d * d);
  }
}

void lagrange_eval(const double* xs, int n, double x, double* out) {
  for (int k = 0; k < n; ++k) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != k) v *= (x - xs[m]) / (xs[k] - xs[m]);
    out[k] = v;
  }
}

void lagrange_deriv_eval(const double* xs, int n, double x, double* out) {
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == k) continue;
      double t = 1.0 / (xs[k] - xs[j]);
      for (int m = 0; m < n; ++m)
        if (m != k && m != j) t *= (x - xs[m]) / (xs[k] - xs[m]);
      s += t;
    }
    out[k] = s;
  }
}

void build_basis(int p, BasisTab<double>& t) {
  std::memset(&t, 0, sizeof(t));
  const int P = p + 1;
  gauss_legendre(P, t.x, t.w);
  for (int i = 0; i < P; ++i) lagrange_deriv_eval(t.x, P, t.x[i], t.D[i]);
  lagrange_eval(t.x, P, -1.0, t.ext[0]);
  lagrange_eval(t.x, P, 1.0, t.ext[1]);
  lagrange_deriv_eval(t.x, P, -1.0, t.dext[0]);
  lagrange_deriv_eval(t.x, P, 1.0, t.dext[1]);
  // g_L = (-1)^p/2 (P_p - P_{p+1}),  g_R = (P_p + P_{p+1})/2
  const double sgn = (p % 2 == 0) ? 1.0 : -1.0;
  for (int i = 0; i < P; ++i) {
    double a = legendre_dp(p, t.x[i]), b = legendre_dp(p + 1, t.x[i]);
    t.dg[0][i] = 0.5 * sgn * (a - b);
    t.dg[1][i] = 0.5 * (a + b);
  }
  t.dgf[0] = 0.5 * sgn * (legendre_dp(p, -1.0) - legendre_dp(p + 1, -1.0));
  t.dgf[1] = 0.5 * (legendre_dp(p, 1.0) + legendre_dp(p + 1, 1.0));
  for (int i = 0; i < P; ++i)
    for (int k = 0; k < P; ++k) t.Dh[i][k] = t.D[i][k] - t.dg[0][i] * t.ext[0][k] - t.dg[1][i] * t.ext[1][k];
  // modal transform by Gauss quadrature: c_m = (2m+1)/2 sum_i w_i P_m(x_i) s_i
  for (int m = 0; m < P; ++m)
    for (int i = 0; i < P; ++i) {
      double Pm = legendre_p(m, t.x[i]);
      t.modal[m][i] = 0.5 * (2 * m + 1) * t.w[i] * Pm;
      t.nodal[i][m] = Pm;
    }
}

void build_mortar(int ps, int pm, MortarTab<double>& t) {
  std::memset(&t, 0, sizeof(t));
  const int Ps = ps + 1, Pm = pm + 1;
  double xs[kPM], ws[kPM], xm[kPM], wm[kPM];
  gauss_legendre(Ps, xs, ws);
  gauss_legendre(Pm, xm, wm);
  for (int m = 0; m < Pm; ++m) lagrange_eval(xs, Ps, xm[m], t.I[m]);
  for (int a = 0; a < Ps; ++a)
    for (int m = 0; m < Pm; ++m) t.Pi[a][m] = wm[m] * t.I[m][a] / ws[a];
}

}  // namespace frgb
