// The Davidson subspace eigenproblem and the biorthonormalisation inverse in FP64 on the GPU.
//
// One warp solves one small dense problem (m <= a few hundred): the 32 lanes share the
// row and column updates of each step, the scalar decisions (shifts, deflation) are taken
// identically by every lane.  The algorithms are the textbook ones: Householder reduction to
// upper Hessenberg form, shifted QR iterations with Givens rotations in complex arithmetic
// (Wilkinson shift from the trailing 2 x 2 block, an exceptional shift every 11 iterations),
// inverse iteration for a real eigenvector, and LU with partial pivoting.
#include <cuda_runtime.h>

#include <cmath>
#include <stdexcept>
#include <string>

#include "kernels.cuh"
#include "subspace.h"

namespace ccsd {
namespace {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx mk(double r, double i = 0.0) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cplx operator*(double s, cplx a) { return mk(s * a.re, s * a.im); }
__device__ __forceinline__ cplx conj(cplx a) { return mk(a.re, -a.im); }
__device__ __forceinline__ double norm2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ double cabs(cplx a) { return hypot(a.re, a.im); }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  const double d = norm2(b);
  return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ cplx csqrt(cplx a) {
  const double r = cabs(a);
  const double x = sqrt(0.5 * (r + fabs(a.re)));
  if (x == 0.0) return mk(0.0);
  const double y = a.im / (2.0 * x);
  return a.re >= 0.0 ? mk(x, y) : mk(fabs(y), a.im >= 0.0 ? x : -x);
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ cplx warp_sum(cplx x) { return mk(warp_sum(x.re), warp_sum(x.im)); }

// Householder reduction of H (n x n, row-major, complex) to upper Hessenberg form; u is n scratch.
__device__ void hessenberg(int n, cplx* H, cplx* u) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 2 < n; ++k) {
    double a2 = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) a2 += norm2(H[i * n + k]);
    const double alpha = sqrt(warp_sum(a2));
    if (alpha == 0.0) continue;
    const cplx x0 = H[(k + 1) * n + k];
    const double ax0 = cabs(x0);
    const cplx phase = ax0 > 0.0 ? mk(x0.re / ax0, x0.im / ax0) : mk(1.0);
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) u[i] = (i == k + 1) ? x0 + alpha * phase : H[i * n + k];
    __syncwarp();
    double un = 0.0;
    for (int i = k + 1 + lane; i < n; i += 32) un += norm2(u[i]);
    un = warp_sum(un);
    if (un == 0.0) continue;
    // H <- (I - 2 u u^H / un) H: column j by lane
    for (int j = lane; j < n; j += 32) {
      cplx s = mk(0.0);
      for (int i = k + 1; i < n; ++i) s = s + conj(u[i]) * H[i * n + j];
      s = (2.0 / un) * s;
      for (int i = k + 1; i < n; ++i) H[i * n + j] = H[i * n + j] - u[i] * s;
    }
    __syncwarp();
    // H <- H (I - 2 u u^H / un): row i by lane
    for (int i = lane; i < n; i += 32) {
      cplx s = mk(0.0);
      for (int j = k + 1; j < n; ++j) s = s + H[i * n + j] * u[j];
      s = (2.0 / un) * s;
      for (int j = k + 1; j < n; ++j) H[i * n + j] = H[i * n + j] - s * conj(u[j]);
    }
    __syncwarp();
  }
}

// All eigenvalues of the real n x n matrix A (leading dimension lda) into ev[n] (order of
// deflation); H is n*n complex scratch, cs/sn n each.
__device__ void eigenvalues(int n, const double* A, int lda, cplx* H, cplx* u, cplx* cs, cplx* sn, cplx* ev) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < n * n; e += 32) H[e] = mk(A[(e / n) * lda + e % n]);
  __syncwarp();
  hessenberg(n, H, u);
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, nev = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev[nev++] = H[0];
      break;
    }
    int lo = hi;
    while (lo > 0) {
      double s = cabs(H[lo * n + lo]) + cabs(H[(lo - 1) * n + lo - 1]);
      if (s == 0.0) s = 1.0;
      if (cabs(H[lo * n + lo - 1]) <= eps * s) break;
      --lo;
    }
    __syncwarp();
    if (lo > 0 && lane == 0) H[lo * n + lo - 1] = mk(0.0);
    __syncwarp();
    if (lo == hi) {
      ev[nev++] = H[hi * n + hi];
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 200 * n) {  // no convergence: the diagonal
      for (int i = hi; i >= 0; --i) ev[nev++] = H[i * n + i];
      break;
    }
    const cplx a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi], c = H[hi * n + hi - 1], d = H[hi * n + hi];
    const cplx tr = a + d, det = a * d - b * c;
    const cplx disc = csqrt(0.25 * (tr * tr) - det);
    const cplx l1 = 0.5 * tr + disc, l2 = 0.5 * tr - disc;
    cplx mu = (cabs(l1 - d) < cabs(l2 - d)) ? l1 : l2;
    if (iter % 11 == 10) mu = mu + mk(cabs(H[hi * n + hi - 1]));
    __syncwarp();
    for (int k = lo + lane; k <= hi; k += 32) H[k * n + k] = H[k * n + k] - mu;
    __syncwarp();
    // H - mu = Q R by Givens rotations of rows k, k+1 (columns shared by the lanes)
    for (int k = lo; k < hi; ++k) {
      const cplx x = H[k * n + k], y = H[(k + 1) * n + k];
      const double r = sqrt(norm2(x) + norm2(y));
      const cplx cc = (r == 0.0) ? mk(1.0) : mk(x.re / r, x.im / r);
      const cplx ss = (r == 0.0) ? mk(0.0) : mk(y.re / r, y.im / r);
      __syncwarp();
      if (lane == 0) {
        cs[k - lo] = cc;
        sn[k - lo] = ss;
      }
      for (int j = k + lane; j < n; j += 32) {
        const cplx t1 = H[k * n + j], t2 = H[(k + 1) * n + j];
        H[k * n + j] = conj(cc) * t1 + conj(ss) * t2;
        H[(k + 1) * n + j] = mk(0.0) - ss * t1 + cc * t2;
      }
      __syncwarp();
    }
    // H <- R Q (columns k, k+1, rows shared by the lanes)
    for (int k = lo; k < hi; ++k) {
      const cplx cc = cs[k - lo], ss = sn[k - lo];
      const int top = min(k + 2, hi);
      for (int i = lane; i <= top; i += 32) {
        const cplx t1 = H[i * n + k], t2 = H[i * n + k + 1];
        H[i * n + k] = t1 * cc + t2 * ss;
        H[i * n + k + 1] = mk(0.0) - t1 * conj(ss) + t2 * conj(cc);
      }
      __syncwarp();
    }
    for (int k = lo + lane; k <= hi; k += 32) H[k * n + k] = H[k * n + k] + mu;
    __syncwarp();
  }
}

// LU with partial pivoting of M (n x n, row-major, in place) and solve for b in place;
// false if singular.  piv is n scratch.
__device__ bool lu_solve(int n, double* M, int* piv, double* b) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < n; ++k) {
    // pivot: the largest |M[i][k]|, i >= k (first one on ties)
    double best = -1.0;
    int p = k;
    for (int i = k + lane; i < n; i += 32) {
      const double v = fabs(M[i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) {
        best = ob;
        p = op;
      }
    }
    if (best == 0.0) return false;
    if (lane == 0) piv[k] = p;
    if (p != k) {
      for (int j = lane; j < n; j += 32) {
        const double t = M[k * n + j];
        M[k * n + j] = M[p * n + j];
        M[p * n + j] = t;
      }
      if (lane == 0) {
        const double t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
    __syncwarp();
    const double d = M[k * n + k];
    for (int i = k + 1 + lane; i < n; i += 32) {
      const double f = M[i * n + k] / d;
      M[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
      b[i] -= f * b[k];
    }
    __syncwarp();
  }
  // back substitution (the dot products shared by the lanes)
  for (int i = n - 1; i >= 0; --i) {
    double s = 0.0;
    for (int j = i + 1 + lane; j < n; j += 32) s += M[i * n + j] * b[j];
    s = warp_sum(s);
    __syncwarp();
    if (lane == 0) b[i] = (b[i] - s) / M[i * n + i];
    __syncwarp();
  }
  return true;
}

// Right eigenvector of A (n x n, lda) for the real eigenvalue lam by inverse iteration with a
// tiny shift; unit 2-norm.  M is n*n scratch, piv n, x and y n each.
__device__ void eigenvector(int n, const double* A, int lda, double lam, double* M, int* piv, double* x, double* y) {
  const int lane = threadIdx.x & 31;
  double sc = 0.0;
  for (int e = lane; e < n * n; e += 32) sc = fmax(sc, fabs(A[(e / n) * lda + e % n]));
  for (int o = 16; o > 0; o >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
  if (sc == 0.0) sc = 1.0;
  double shift = lam + 1e-13 * sc;
  for (int i = lane; i < n; i += 32) x[i] = 1.0 + 0.01 * i;
  __syncwarp();
  for (int it = 0; it < 4; ++it) {
    bool ok = false;
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
      for (int e = lane; e < n * n; e += 32) M[e] = A[(e / n) * lda + e % n] - ((e / n == e % n) ? shift : 0.0);
      for (int i = lane; i < n; i += 32) y[i] = x[i];
      __syncwarp();
      ok = lu_solve(n, M, piv, y);
      if (!ok) shift += 1e-12 * sc;
    }
    if (!ok) break;
    double nn = 0.0;
    for (int i = lane; i < n; i += 32) nn += y[i] * y[i];
    const double nrm = sqrt(warp_sum(nn));
    if (nrm == 0.0 || !isfinite(nrm)) break;
    __syncwarp();
    for (int i = lane; i < n; i += 32) x[i] = y[i] / nrm;
    __syncwarp();
  }
}

// One warp: the subspace step of the Davidson solver (see subspace.h).
__global__ void k_subspace_step(int m, const double* __restrict__ G, int ldg, int nroots,
                                const double* __restrict__ targets, double* __restrict__ out, double* work) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  cplx* H = reinterpret_cast<cplx*>(work);
  cplx* u = H + m * m;
  cplx* cs = u + m;
  cplx* sn = cs + m;
  cplx* ev = sn + m;
  double* M = reinterpret_cast<double*>(ev + m);
  double* x = M + m * m;
  double* y = x + m;
  double* prev = y + m;
  int* piv = reinterpret_cast<int*>(prev + m);
  int* used = piv + m;
  int* sel = used + m;
  eigenvalues(m, G, ldg, H, u, cs, sn, ev);
  __syncwarp();
  // sort by real part (insertion sort, lane 0)
  if (lane == 0) {
    for (int i = 1; i < m; ++i) {
      const cplx key = ev[i];
      int j = i - 1;
      while (j >= 0 && ev[j].re > key.re) {
        ev[j + 1] = ev[j];
        --j;
      }
      ev[j + 1] = key;
    }
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = fmax(scale, cabs(ev[i]));
    // wanted roots: the lowest by real part, or the ones nearest the targets
    for (int i = 0; i < m; ++i) used[i] = 0;
    for (int k = 0; k < nroots; ++k) {
      int best = k;
      if (targets) {
        best = -1;
        for (int q = 0; q < m; ++q)
          if (!used[q] && (best < 0 || fabs(ev[q].re - targets[k]) < fabs(ev[best].re - targets[k]))) best = q;
        used[best] = 1;
      }
      sel[k] = best;
    }
    out[2 * nroots + m * nroots] = scale;
  }
  __syncwarp();
  const double scale = out[2 * nroots + m * nroots];
  const double tiny = 1e-9 * fmax(scale, 1.0);
  bool have_prev = false;
  double prev_re = 0.0;
  for (int k = 0; k < nroots; ++k) {
    const cplx e = ev[sel[k]];
    const bool is_c = fabs(e.im) > tiny;
    const bool partner = is_c && k > 0 && have_prev && fabs(e.re - prev_re) <= 1e-12 * fmax(scale, 1.0);
    if (partner) {  // (G - a) u_prev, normalised: the second vector of the pair's real invariant subspace
      for (int i = lane; i < m; i += 32) {
        double s = -e.re * prev[i];
        for (int j = 0; j < m; ++j) s += G[i * ldg + j] * prev[j];
        y[i] = s;
      }
      double nn = 0.0;
      for (int i = lane; i < m; i += 32) nn += y[i] * y[i];
      const double nrm = sqrt(fmax(warp_sum(nn), 1e-300));
      __syncwarp();
      for (int i = lane; i < m; i += 32) out[2 * nroots + i * nroots + k] = y[i] / nrm;
      have_prev = false;
    } else {
      eigenvector(m, G, ldg, e.re, M, piv, x, y);
      __syncwarp();
      for (int i = lane; i < m; i += 32) {
        out[2 * nroots + i * nroots + k] = x[i];
        if (is_c) prev[i] = x[i];
      }
      have_prev = is_c;
      prev_re = e.re;
    }
    if (lane == 0) {
      out[k] = e.re;
      out[nroots + k] = e.im;
    }
    __syncwarp();
  }
}

// One warp: Minv = M^-1 for an n x n matrix (row-major), flag[0] = 1 if singular.
__global__ void k_small_inverse(int n, const double* __restrict__ A, double* __restrict__ Ainv, int* flag,
                                double* work) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double* M = work;
  double* b = M + n * n;
  int* piv = reinterpret_cast<int*>(b + n);
  if (lane == 0) flag[0] = 0;
  for (int col = 0; col < n; ++col) {
    for (int e = lane; e < n * n; e += 32) M[e] = A[e];
    for (int i = lane; i < n; i += 32) b[i] = (i == col) ? 1.0 : 0.0;
    __syncwarp();
    if (!lu_solve(n, M, piv, b)) {
      if (lane == 0) flag[0] = 1;
      return;
    }
    for (int r = lane; r < n; r += 32) Ainv[r * n + col] = b[r];
    __syncwarp();
  }
}

}  // namespace

size_t subspace_work_bytes(int m) { return (size_t)(m * m + 4 * m) * 16 + (size_t)(m * m + 3 * m) * 8 + (size_t)3 * m * 4 + 64; }

void launch_subspace_step(int m, const double* G, int ldg, int nroots, const double* targets, double* out, void* work,
                          cudaStream_t st) {
  if (m < 1 || nroots < 1 || nroots > m) throw std::runtime_error("subspace step: bad sizes");
  count_launches(1);
  k_subspace_step<<<1, 32, 0, st>>>(m, G, ldg, nroots, targets, out, (double*)work);
}

size_t small_inverse_work_bytes(int n) { return (size_t)(n * n + n) * 8 + (size_t)n * 4 + 64; }

void launch_small_inverse(int n, const double* A, double* Ainv, int* flag, void* work, cudaStream_t st) {
  if (n < 1) throw std::runtime_error("small inverse: bad size");
  count_launches(1);
  k_small_inverse<<<1, 32, 0, st>>>(n, A, Ainv, flag, (double*)work);
}

}  // namespace ccsd
