// FP64-grade products on the tensor cores (fp64_tc.cu): fixed-point bf16 slices
// whose per-chunk FP32 sums are exact, read out into 64-bit integer accumulators.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "kernels.cuh"

namespace ccsd {
namespace oz {

constexpr int S = 7;          // 7-bit slices per operand (49 bits below the row's leading bit)
constexpr int NPROD = 28;     // slice products a_s b_t with s + t <= 6
constexpr int BN = 64;        // output tile 128 x 64
constexpr int KC_TILES = 8;   // K chunk between accumulator read-outs: 8 x 64 = 512
constexpr int NONFINITE = 100000;  // row exponent marking a row with Inf or NaN

// Device bytes of one operand: S bf16 planes [S][rows_p][Kp] followed by rows_p int row exponents.
size_t operand_bytes(int64_t rows_p, int64_t Kp);
inline int* exps_of(void* buf, int64_t rows_p, int64_t Kp) {
  return (int*)((char*)buf + (size_t)S * rows_p * Kp * 2);
}

// Fill buf (operand_bytes(rows_p, Kp)) from the FP64 operand given as a strided gather
// over (row dims..., K dims...) with source strides in g.s1; padding rows and K are zero.
void pack(cudaStream_t st, const double* src, const Strided& g, int64_t rows, int64_t rows_p, int64_t K, int64_t Kp,
          void* buf);

// C = alpha A B^T + beta C (beta 0 or 1) from packed operands: a with Mp rows (multiple of 128),
// b with Np rows (multiple of BN), Kp (multiple of 64).  Output (m, n) at C + m sCm + n sCn, or,
// with om and on given, at C + off(m; om) + off(n; on).  nsplit 0: heuristic split-K count.
// err: device flag raised when a wait of the kernel times out.  Returns the MMA flops issued.
double gemm(cudaStream_t st, const void* a, int64_t Mp, const void* b, int64_t Np, int64_t Kp, int M, int N,
            double* C, int64_t sCm, int64_t sCn, double alpha, double beta, const Strided* om, const Strided* on,
            int nsplit, int* err, long long budget);

}  // namespace oz

// C[m, n] = sum_z part[z][m][n] (+ C[m, n] unless beta_zero), output addressed as in oz::gemm
// (tc_gemm.cu).
void launch_split_reduce_fp64(int M, int N, int nsplit, const double* part, double* C, long long sCm, long long sCn,
                              int beta_zero, const Strided* om, const Strided* on, cudaStream_t st);

}  // namespace ccsd
