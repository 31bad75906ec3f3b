// Host-side setup arithmetic: the Vanka stencil coefficients (eq. (6)), the LFA
// choice of the relaxation parameter (eq. (4)-(5)) and dense complex inversion for the
// coarsest grid.
#include <cmath>
#include <complex>
#include <vector>

#include "pd_internal.h"

namespace pd {

using cd = std::complex<double>;

// a, b, c of eq. (6) for eta = lam h^2; out = {Re a, Im a, Re b, Im b, Re c, Im c}.
void vanka_abc(double er, double ei, double out[6]) {
  const cd eta(er, ei);
  const cd p = 1.0 / (2.0 + eta), q = 1.0 / (4.0 + eta), s = 1.0 / (6.0 + eta);
  const cd a = 0.25 * (p + 2.0 * q + s), b = 0.25 * (p - s), c = 0.25 * (p - 2.0 * q + s);
  out[0] = a.real(); out[1] = a.imag();
  out[2] = b.real(); out[3] = b.imag();
  out[4] = c.real(); out[5] = c.imag();
}

// omega_opt = argmin over omega in [0.5, 1.5] of mu_loc = max over the sampled high
// frequencies of |1 - omega M~ L~| (eq. (4)-(5), symbols of Sec. 2.1).  Sampling:
// theta = -pi/2 + 2 pi a / 64 per axis, a = 0..63, a point being high when one
// coordinate lies in [pi/2, 3pi/2).  The symbols depend on cos(theta) only; those
// cosines are cos(2 pi p / 64), p = 0..32, and a pair is high exactly when one of its
// p lies in [16, 32], so the maximum runs over those pairs.  mu_loc is a maximum of
// |1 - omega s| over the samples, convex in real omega: golden-section search.
double lfa_omega_opt(double er, double ei, int jacobi) {
  const cd eta(er, ei);
  double a6[6];
  vanka_abc(er, ei, a6);
  const cd a(a6[0], a6[1]), b(a6[2], a6[3]), c(a6[4], a6[5]);
  double cs[33];
  for (int p = 0; p <= 32; p++) cs[p] = std::cos(2.0 * M_PI * p / 64.0);
  std::vector<cd> sym;
  sym.reserve(33 * 33);
  for (int p = 0; p <= 32; p++)
    for (int q = 0; q <= 32; q++) {
      if (p < 16 && q < 16) continue;
      const double c1 = cs[p], c2 = cs[q];
      const cd Lh = 4.0 + eta - 2.0 * c1 - 2.0 * c2;
      const cd Mh = jacobi ? 1.0 / (4.0 + eta) : a + b * c1 + b * c2 + c * c1 * c2;
      sym.push_back(Mh * Lh);
    }
  auto mu = [&](double w) {
    double m = 0.0;
    for (const cd &s : sym) m = std::fmax(m, std::abs(1.0 - w * s));
    return m;
  };
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double lo = 0.5, hi = 1.5;
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  double f1 = mu(x1), f2 = mu(x2);
  while (hi - lo > 1e-12) {
    if (f1 <= f2) {
      hi = x2; x2 = x1; f2 = f1;
      x1 = hi - g * (hi - lo);
      f1 = mu(x1);
    } else {
      lo = x1; x1 = x2; f1 = f2;
      x2 = lo + g * (hi - lo);
      f2 = mu(x2);
    }
  }
  return 0.5 * (lo + hi);
}

// In-place inverse of the complex m x m matrix A (interleaved re, im, row-major) by
// Gauss-Jordan elimination with partial pivoting.  Returns 0, or -1 if singular.
int invert_dense(int m, std::vector<double> &A) {
  std::vector<cd> M((size_t)m * 2 * m);
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) {
      M[(size_t)i * 2 * m + j] = cd(A[2 * ((size_t)i * m + j)], A[2 * ((size_t)i * m + j) + 1]);
      M[(size_t)i * 2 * m + m + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int k = 0; k < m; k++) {
    int p = k;
    for (int i = k + 1; i < m; i++)
      if (std::abs(M[(size_t)i * 2 * m + k]) > std::abs(M[(size_t)p * 2 * m + k])) p = i;
    if (std::abs(M[(size_t)p * 2 * m + k]) == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < 2 * m; j++) std::swap(M[(size_t)k * 2 * m + j], M[(size_t)p * 2 * m + j]);
    const cd piv = 1.0 / M[(size_t)k * 2 * m + k];
    for (int j = 0; j < 2 * m; j++) M[(size_t)k * 2 * m + j] *= piv;
    for (int i = 0; i < m; i++) {
      if (i == k) continue;
      const cd f = M[(size_t)i * 2 * m + k];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * m; j++) M[(size_t)i * 2 * m + j] -= f * M[(size_t)k * 2 * m + j];
    }
  }
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) {
      const cd v = M[(size_t)i * 2 * m + m + j];
      A[2 * ((size_t)i * m + j)] = v.real();
      A[2 * ((size_t)i * m + j) + 1] = v.imag();
    }
  return 0;
}

}  // namespace pd
