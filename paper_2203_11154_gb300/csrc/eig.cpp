// Eigendecomposition B = V D V^{-1} of a real time matrix (Sec. 1: the diagonalisation
// that turns the all-at-once system (1) into the shifted systems (2)), on the host at
// set-up, for any diagonalisable B with distinct eigenvalues (e.g. the boundary-value
// B of Example 1, eq. (9), or the quasi-BVM B of Example 2, eq. (10)).
//
// Steps (standard dense nonsymmetric eigenvalue algorithm):
//   1. balancing by powers of two, B' = D^{-1} B D (Parlett & Reinsch, 1969), which
//      evens out row and column norms (Example 2's 1/beta corner) without rounding;
//   2. Householder reduction to upper Hessenberg form, B' = Q H Q^T;
//   3. complex Schur form H = Z T Z^H by shifted QR steps (Givens rotations, Wilkinson
//      shift from the trailing 2 x 2 block, an exceptional shift after every 10 steps
//      without deflation, deflation when a subdiagonal entry drops below eps times its
//      diagonal neighbours);
//   4. eigenvectors of the triangular T by back substitution, (T - t_kk I) y = 0 with
//      y_k = 1, mapped back as v = D Q Z y and scaled to unit 2-norm;
//   5. V^{-1} by Gauss-Jordan elimination with partial pivoting; a condition number of V
//      beyond 1/(64 eps) (a defective B) is an error.
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "pd_internal.h"

namespace pd {

namespace {

using cd = std::complex<double>;

// Parlett-Reinsch balancing of the real n x n row-major A in place; d receives the
// diagonal scaling (A <- D^{-1} A D).  Scale factors are powers of two (exact).
void balance(int n, std::vector<double> &A, std::vector<double> &d) {
  d.assign(n, 1.0);
  const double radix = 2.0, r2 = radix * radix;
  bool done = false;
  for (int sweep = 0; !done && sweep < 100; sweep++) {
    done = true;
    for (int i = 0; i < n; i++) {
      double c = 0.0, r = 0.0;
      for (int j = 0; j < n; j++)
        if (j != i) {
          c += std::fabs(A[(size_t)j * n + i]);
          r += std::fabs(A[(size_t)i * n + j]);
        }
      if (c == 0.0 || r == 0.0) continue;
      double g = r / radix, f = 1.0;
      const double s = c + r;
      while (c < g) {
        f *= radix;
        c *= r2;
      }
      g = r * radix;
      while (c > g) {
        f /= radix;
        c /= r2;
      }
      if ((c + r) / f < 0.95 * s) {
        done = false;
        d[i] *= f;
        for (int j = 0; j < n; j++) A[(size_t)i * n + j] /= f;
        for (int j = 0; j < n; j++) A[(size_t)j * n + i] *= f;
      }
    }
  }
}

// Householder reduction of the real n x n A to upper Hessenberg form in place;
// Q (row-major, orthogonal) accumulates the reflections: A_in = Q A_out Q^T.
void hessenberg(int n, std::vector<double> &A, std::vector<double> &Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) Q[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; k++) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; i++) alpha += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = A[(size_t)(k + 1) * n + k];
    if (x0 > 0) alpha = -alpha;  // v = x - alpha e1 without cancellation
    double vn = 0.0;
    for (int i = k + 1; i < n; i++) {
      v[i] = A[(size_t)i * n + k] - (i == k + 1 ? alpha : 0.0);
      vn += v[i] * v[i];
    }
    if (vn == 0.0) continue;
    // A <- (I - 2 v v^T / vn) A (I - 2 v v^T / vn), Q <- Q (I - 2 v v^T / vn)
    for (int j = 0; j < n; j++) {
      double s = 0.0;
      for (int i = k + 1; i < n; i++) s += v[i] * A[(size_t)i * n + j];
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; i++) A[(size_t)i * n + j] -= s * v[i];
    }
    for (int i = 0; i < n; i++) {
      double s = 0.0, q = 0.0;
      for (int j = k + 1; j < n; j++) {
        s += A[(size_t)i * n + j] * v[j];
        q += Q[(size_t)i * n + j] * v[j];
      }
      s *= 2.0 / vn;
      q *= 2.0 / vn;
      for (int j = k + 1; j < n; j++) {
        A[(size_t)i * n + j] -= s * v[j];
        Q[(size_t)i * n + j] -= q * v[j];
      }
    }
    for (int i = k + 2; i < n; i++) A[(size_t)i * n + k] = 0.0;
  }
}

// Givens rotation [c s; -conj(s) c] (c real) with [c s; -conj(s) c] [a; b] = [r; 0].
void givens(cd a, cd b, double &c, cd &s) {
  const double aa = std::abs(a), bb = std::abs(b);
  if (bb == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (aa == 0.0) {
    c = 0.0;
    s = std::conj(b) / bb;
    return;
  }
  const double nrm = std::hypot(aa, bb);
  c = aa / nrm;
  s = (a / aa) * std::conj(b) / nrm;
}

// Complex Schur form of the Hessenberg T (n x n, row-major, in place): T <- Z^H T Z upper
// triangular, Z accumulated (Z <- Z G).  Returns false if the iteration does not settle.
bool schur(int n, std::vector<cd> &T, std::vector<cd> &Z) {
  const double eps = std::numeric_limits<double>::epsilon();
  double tnorm = 0.0;
  for (const cd &x : T) tnorm = std::fmax(tnorm, std::abs(x));
  if (tnorm == 0.0) return true;
  auto at = [&](int i, int j) -> cd & { return T[(size_t)i * n + j]; };
  std::vector<double> gc(n);
  std::vector<cd> gs(n);
  int hi = n - 1, iter = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    for (; l > 0; l--) {
      double s = std::abs(at(l - 1, l - 1)) + std::abs(at(l, l));
      if (s == 0.0) s = tnorm;
      if (std::abs(at(l, l - 1)) <= eps * s) {
        at(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == hi) {
      hi--;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    iter++;
    cd mu;
    if (iter % 10 == 0) {
      // exceptional shift: breaks cycles of the Wilkinson shift
      const double ex = std::abs(at(hi, hi - 1)) + (hi - 2 >= l ? std::abs(at(hi - 1, hi - 2)) : 0.0);
      mu = at(hi, hi) + cd(0.75 * ex, 0.0);
    } else {
      const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
      const cd half = 0.5 * (a - d);
      const cd disc = std::sqrt(half * half + b * c);
      const cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = std::abs(m1 - d) <= std::abs(m2 - d) ? m1 : m2;
    }
    // explicit shifted QR step on the active block [l, hi] of the whole matrix
    for (int k = l; k <= hi; k++) at(k, k) -= mu;
    for (int k = l; k < hi; k++) {
      givens(at(k, k), at(k + 1, k), gc[k], gs[k]);
      const double c = gc[k];
      const cd s = gs[k];
      for (int j = k; j < n; j++) {
        const cd x = at(k, j), y = at(k + 1, j);
        at(k, j) = c * x + s * y;
        at(k + 1, j) = -std::conj(s) * x + c * y;
      }
    }
    for (int k = l; k < hi; k++) {
      const double c = gc[k];
      const cd s = gs[k];
      // right multiplication by G^H: columns k, k+1
      for (int i = 0; i <= std::min(k + 1, hi); i++) {
        const cd x = at(i, k), y = at(i, k + 1);
        at(i, k) = c * x + std::conj(s) * y;
        at(i, k + 1) = -s * x + c * y;
      }
      for (int i = 0; i < n; i++) {
        cd &x = Z[(size_t)i * n + k], &y = Z[(size_t)i * n + k + 1];
        const cd zx = x, zy = y;
        x = c * zx + std::conj(s) * zy;
        y = -s * zx + c * zy;
      }
    }
    for (int k = l; k <= hi; k++) at(k, k) += mu;
  }
  for (int i = 1; i < n; i++)
    for (int j = 0; j < i; j++) at(i, j) = 0.0;
  return true;
}

}  // namespace

int diagonalize(int n, const double *B, std::vector<double> &lam, std::vector<double> &V,
                std::vector<double> &Vinv) {
  if (n < 1) return -1;
  for (size_t e = 0; e < (size_t)n * n; e++)
    if (!std::isfinite(B[e])) return -1;
  std::vector<double> A(B, B + (size_t)n * n), d, Q;
  balance(n, A, d);
  hessenberg(n, A, Q);
  std::vector<cd> T((size_t)n * n), Z((size_t)n * n);
  for (size_t e = 0; e < (size_t)n * n; e++) {
    T[e] = A[e];
    Z[e] = Q[e];
  }
  if (!schur(n, T, Z)) return -2;
  double tnorm = 0.0;
  for (const cd &x : T) tnorm = std::fmax(tnorm, std::abs(x));
  const double small = std::fmax(std::numeric_limits<double>::epsilon() * tnorm,
                                 std::numeric_limits<double>::min());
  lam.assign(2 * (size_t)n, 0.0);
  V.assign(2 * (size_t)n * n, 0.0);
  std::vector<cd> y(n), v(n);
  for (int k = 0; k < n; k++) {
    const cd tk = T[(size_t)k * n + k];
    lam[2 * k] = tk.real();
    lam[2 * k + 1] = tk.imag();
    for (int i = 0; i < n; i++) y[i] = 0.0;
    y[k] = 1.0;
    for (int i = k - 1; i >= 0; i--) {
      cd s = 0.0;
      for (int j = i + 1; j <= k; j++) s += T[(size_t)i * n + j] * y[j];
      cd dd = T[(size_t)i * n + i] - tk;
      if (std::abs(dd) < small) dd = small;
      y[i] = -s / dd;
      // keep the entries representable (rescaling does not change the direction)
      const double big = std::abs(y[i]);
      if (big > 1e100)
        for (int j = i; j <= k; j++) y[j] /= big;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; i++) {
      cd s = 0.0;
      for (int j = 0; j <= k; j++) s += Z[(size_t)i * n + j] * y[j];
      v[i] = d[i] * s;
      nrm += std::norm(v[i]);
    }
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return -3;
    for (int i = 0; i < n; i++) {
      V[2 * ((size_t)i * n + k)] = v[i].real() / nrm;
      V[2 * ((size_t)i * n + k) + 1] = v[i].imag() / nrm;
    }
  }
  Vinv = V;
  if (invert_dense(n, Vinv) != 0) return -4;
  // a defective B (no basis of eigenvectors) leaves V singular up to rounding: reject a
  // 1-norm condition number beyond what FP64 can resolve
  double n1 = 0.0, ni1 = 0.0;
  for (int j = 0; j < n; j++) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < n; i++) {
      const size_t e = (size_t)i * n + j;
      a += std::hypot(V[2 * e], V[2 * e + 1]);
      b += std::hypot(Vinv[2 * e], Vinv[2 * e + 1]);
    }
    n1 = std::fmax(n1, a);
    ni1 = std::fmax(ni1, b);
  }
  if (!(n1 * ni1 <= 1.0 / (64.0 * std::numeric_limits<double>::epsilon()))) return -5;
  return 0;
}

}  // namespace pd
