// CUDA kernels of the CCSD library (sm_103a).  All arithmetic here is FP64
// unless stated; the tensor-core GEMM lives in tc_gemm.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccsd {

constexpr int kMaxDims = 8;

// Number of kernels this library has launched (all streams, all handles).
long long kernel_launches();
void count_launches(int n);

// A strided index space: ndim dims with extents, plus per-dim strides of up to
// two addressed arrays.  Linear index -> row-major coordinates over ext.
struct Strided {
  int ndim = 0;
  int64_t ext[kMaxDims];
  int64_t s0[kMaxDims];  // strides of array 0
  int64_t s1[kMaxDims];  // strides of array 1
  int64_t total() const {
    int64_t t = 1;
    for (int d = 0; d < ndim; ++d) t *= ext[d];
    return t;
  }
};

// dst (strides s0) += alpha * src (strides s1) over the index space; dst
// elements must be distinct (no two indices address the same dst element).
void launch_axpy_strided(double* dst, const double* src, const Strided& sp, double alpha, cudaStream_t st);
// dst (strides s0) = src (strides s1) over the index space.
void launch_copy_strided(double* dst, const double* src, const Strided& sp, cudaStream_t st);
// dst (strides s0) = 0 over the index space.
void launch_zero_strided(double* dst, const Strided& sp, cudaStream_t st);

// Batched FP64 GEMM with arbitrary element strides:
//   C[b][m][n] = alpha * sum_k A[b][m][k] B[b][n][k] + beta * C[b][m][n]
struct GemmArgs {
  int batch, M, N, K;
  const double* A;
  int64_t sAb, sAm, sAk;
  const double* B;
  int64_t sBb, sBn, sBk;
  double* C;
  int64_t sCb, sCm, sCn;
  double alpha, beta;
};
void launch_dgemm(const GemmArgs& g, cudaStream_t st);

// ---- amplitude-vector kernels (vector = o*v singles [i][a] + o*o*v*v doubles [i][j][a][b]) ----
struct VecShape {
  int o, v;
  __host__ __device__ int64_t n1() const { return (int64_t)o * v; }
  __host__ __device__ int64_t dim() const { return n1() + (int64_t)o * o * v * v; }
};

// G[p*ldg + q] = <X_p | Y_q> (packed inner product: doubles weighted 1/2, 1 on the
// diagonal ai = bj) for p < np, q < nq; X_p = X + p*ldx, Y_q = Y + q*ldy.
// `work` must hold at least wdot_work_size(np, nq) doubles.
int64_t wdot_work_size(int np, int nq);
void launch_wdot(const VecShape& s, const double* X, int64_t ldx, int np, const double* Y, int64_t ldy, int nq,
                 double* G, int ldg, double* work, cudaStream_t st);
// y_q = sum_p c[p*ldc + q] x_p (+ y_q if accumulate), q < nq.  c is a device array.  FP64, or
// with fp64grade in double-float arithmetic on the FP32 pipe (about 2^-44 of sum_p |c x_p|; for
// coefficients that do not cancel strongly, such as Ritz-vector components).
void launch_lincomb(const VecShape& s, const double* X, int64_t ldx, int np, const double* c, int ldc, double* Y,
                    int64_t ldy, int nq, bool accumulate, cudaStream_t st, bool fp64grade = false);
// y = a*x + b*y over n elements.
void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
// y = x / (D - shift) with D_ai = e_a - e_i, D_aibj = e_a + e_b - e_i - e_j.
void launch_precond(const VecShape& s, const double* eps, const double* x, double* y, double shift,
                    cudaStream_t st);
// doubles *= pair weight (1/2 off the diagonal ai = bj, 1 on it); singles unchanged.
void launch_weight(const VecShape& s, const double* x, double* y, int nvec, int64_t ld, cudaStream_t st);
// derivative w.r.t. packed doubles: y2 = g2 + g2^T (pair transpose), diagonal kept as g2.
void launch_packed_grad(const VecShape& s, const double* g, double* y, int nvec, int64_t ld, cudaStream_t st);
// out[0] = max |x| over n elements (FP64), two-pass through `work` (>= 1024 doubles).
void launch_maxabs(int64_t n, const double* x, double* out, double* work, cudaStream_t st);
// out[0] = index of the first element of largest magnitude (as double), out[1] = that element.
void launch_argmaxabs(int64_t n, const double* x, double* out, double* work, cudaStream_t st);
// t-eta first term: <L|tau_sigma|(r0 + R)> for all packed sigma (see capi.cpp).
void launch_tau_expectation(const VecShape& s, double r0, const double* L, const double* R, double* y,
                            cudaStream_t st);
// out[0] = the biorthonormal-bra metric of a (1/2 sum a_1^2 + sum (2 A^2 + A A_swap(ab))/12
// + 3/4 sum over the diagonal ai = bj), two-pass through work (>= 512 doubles).
void launch_bra_metric(const VecShape& s, const double* a, double* out, double* work, cudaStream_t st);
// x = (t1, t2 - t1 (x) t1): singles copied, doubles t2[i][j][a][b] - t1[i][a] t1[j][b].
void launch_t2_minus_t1t1(const VecShape& s, const double* t, double* x, cudaStream_t st);
// out[p][q] = (D[p][q] - D[q][p]) / 2 for an n x n matrix (out must not overlap D).
void launch_antisymmetric_part(int n, const double* D, double* out, cudaStream_t st);

// Branching plane of two states k < l from their energy gradients gk, gl and the coupling
// f = F_kl along n directions, gap = E_l - E_k (one CTA, FP64):
//   out[0..n)   g = gl - gk
//   out[n..2n)  h = gap * f
//   out[2n..3n) G = P gl + 2 gap g/|g|, P the projector onto the complement of span{g, h}
// (the crossing-point direction of Bearpark, Robb and Schlegel).  out must not overlap the inputs.
void launch_branching_plane(int n, double gap, const double* gk, const double* gl, const double* f, double* out,
                            cudaStream_t st);
// out[0] = sum_k x[k] y[k] over n elements (plain dot), two-pass via work (>= 1024 doubles).
void launch_dot(int64_t n, const double* x, const double* y, double* out, double* work, cudaStream_t st);

}  // namespace ccsd
