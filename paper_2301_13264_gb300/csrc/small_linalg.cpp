#include "small_linalg.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace ccsd {

using cd = std::complex<double>;

bool lu_solve(int n, std::vector<double> A, std::vector<double>& b) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) {
        best = std::fabs(A[i * n + k]);
        p = i;
      }
    if (best == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return true;
}

bool invert(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
  Ainv.assign(n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    std::vector<double> e(n, 0.0);
    e[c] = 1.0;
    if (!lu_solve(n, A, e)) return false;
    for (int r = 0; r < n; ++r) Ainv[r * n + c] = e[r];
  }
  return true;
}

// Householder reduction to upper Hessenberg form (in place, row-major).
static void hessenberg(int n, std::vector<cd>& H) {
  for (int k = 0; k + 2 < n; ++k) {
    double alpha2 = 0.0;
    for (int i = k + 1; i < n; ++i) alpha2 += std::norm(H[i * n + k]);
    double alpha = std::sqrt(alpha2);
    if (alpha == 0.0) continue;
    cd x0 = H[(k + 1) * n + k];
    cd phase = (std::abs(x0) > 0.0) ? x0 / std::abs(x0) : cd(1.0, 0.0);
    std::vector<cd> u(n, 0.0);
    u[k + 1] = x0 + phase * alpha;
    for (int i = k + 2; i < n; ++i) u[i] = H[i * n + k];
    double un = 0.0;
    for (int i = k + 1; i < n; ++i) un += std::norm(u[i]);
    if (un == 0.0) continue;
    // H <- (I - 2 u u^H / un) H (I - 2 u u^H / un)
    for (int j = 0; j < n; ++j) {
      cd s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(u[i]) * H[i * n + j];
      s *= 2.0 / un;
      for (int i = k + 1; i < n; ++i) H[i * n + j] -= u[i] * s;
    }
    for (int i = 0; i < n; ++i) {
      cd s = 0.0;
      for (int j = k + 1; j < n; ++j) s += H[i * n + j] * u[j];
      s *= 2.0 / un;
      for (int j = k + 1; j < n; ++j) H[i * n + j] -= s * std::conj(u[j]);
    }
  }
}

std::vector<cd> eigenvalues(int n, const std::vector<double>& A) {
  std::vector<cd> H(n * n);
  for (int i = 0; i < n * n; ++i) H[i] = A[i];
  hessenberg(n, H);
  std::vector<cd> ev;
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = n - 1;
  int iter = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev.push_back(H[0]);
      break;
    }
    // find the active block [lo, hi]
    int lo = hi;
    while (lo > 0) {
      double s = std::abs(H[lo * n + lo]) + std::abs(H[(lo - 1) * n + lo - 1]);
      if (s == 0.0) s = 1.0;
      if (std::abs(H[lo * n + lo - 1]) <= eps * s) {
        H[lo * n + lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      ev.push_back(H[hi * n + hi]);
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 200 * n) {  // give up on convergence: return diagonal
      for (int i = hi; i >= 0; --i) ev.push_back(H[i * n + i]);
      break;
    }
    // Wilkinson shift from the trailing 2x2 block
    cd a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi], c = H[hi * n + hi - 1], d = H[hi * n + hi];
    cd tr = a + d, det = a * d - b * c;
    cd disc = std::sqrt(tr * tr / 4.0 - det);
    cd l1 = tr / 2.0 + disc, l2 = tr / 2.0 - disc;
    cd mu = (std::abs(l1 - d) < std::abs(l2 - d)) ? l1 : l2;
    if (iter % 11 == 10) mu += std::abs(H[hi * n + hi - 1]);  // exceptional shift
    // QR step on the block via Givens rotations: H - mu I = Q R, H <- R Q + mu I
    std::vector<cd> cs(hi - lo), sn(hi - lo);
    for (int k = lo; k <= hi; ++k) H[k * n + k] -= mu;
    for (int k = lo; k < hi; ++k) {
      cd x = H[k * n + k], y = H[(k + 1) * n + k];
      double r = std::sqrt(std::norm(x) + std::norm(y));
      cd cc = (r == 0.0) ? cd(1.0) : x / r;
      cd ss = (r == 0.0) ? cd(0.0) : y / r;
      cs[k - lo] = cc;
      sn[k - lo] = ss;
      for (int j = k; j < n; ++j) {
        cd t1 = H[k * n + j], t2 = H[(k + 1) * n + j];
        H[k * n + j] = std::conj(cc) * t1 + std::conj(ss) * t2;
        H[(k + 1) * n + j] = -ss * t1 + cc * t2;
      }
    }
    for (int k = lo; k < hi; ++k) {
      cd cc = cs[k - lo], ss = sn[k - lo];
      for (int i = 0; i <= std::min(k + 2, hi); ++i) {
        cd t1 = H[i * n + k], t2 = H[i * n + k + 1];
        H[i * n + k] = t1 * cc + t2 * ss;
        H[i * n + k + 1] = -t1 * std::conj(ss) + t2 * std::conj(cc);
      }
    }
    for (int k = lo; k <= hi; ++k) H[k * n + k] += mu;
  }
  return ev;
}

std::vector<double> eigenvector(int n, const std::vector<double>& A, double lam) {
  double scale = 0.0;
  for (double x : A) scale = std::max(scale, std::fabs(x));
  if (scale == 0.0) scale = 1.0;
  double shift = lam + 1e-13 * scale;
  std::vector<double> M(A);
  for (int i = 0; i < n; ++i) M[i * n + i] -= shift;
  std::vector<double> x(n, 1.0);
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.01 * i;
  for (int it = 0; it < 4; ++it) {
    std::vector<double> y = x;
    if (!lu_solve(n, M, y)) {
      for (int i = 0; i < n; ++i) M[i * n + i] -= 1e-12 * scale;
      y = x;
      if (!lu_solve(n, M, y)) break;
    }
    double nrm = 0.0;
    for (double v : y) nrm += v * v;
    nrm = std::sqrt(nrm);
    if (nrm == 0.0 || !std::isfinite(nrm)) break;
    for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
  }
  return x;
}

}  // namespace ccsd
