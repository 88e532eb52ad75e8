// FP64 kernels: strided permute/accumulate, batched DFMA GEMM, amplitude-vector
// operations (packed inner products, preconditioner, pair symmetrisation).
#include "kernels.cuh"
#include "fpsplit.cuh"

#include "alloc.h"

#include <algorithm>
#include <atomic>
#include <stdexcept>

namespace ccsd {

static std::atomic<long long> g_launches{0};
long long kernel_launches() { return g_launches.load(); }
void count_launches(int n) { g_launches.fetch_add(n); }

static inline int grid_for(int64_t n, int block = 256, int cap = 152 * 16) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ---------------------------------------------------------------------------
// strided axpy / zero
// ---------------------------------------------------------------------------
template <typename I, bool COPY>
__global__ void k_axpy_strided(double* __restrict__ dst, const double* __restrict__ src, Strided sp, I total,
                               double alpha) {
  for (I idx = (I)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (I)gridDim.x * blockDim.x) {
    I r = idx;
    int64_t o0 = 0, o1 = 0;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      I e = (I)sp.ext[d];
      I c = r % e;
      r /= e;
      o0 += (int64_t)c * sp.s0[d];
      o1 += (int64_t)c * sp.s1[d];
    }
    if (COPY)
      dst[o0] = src[o1];
    else
      dst[o0] += alpha * src[o1];
  }
}

template <typename I>
__global__ void k_zero_strided(double* __restrict__ dst, Strided sp, I total) {
  for (I idx = (I)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (I)gridDim.x * blockDim.x) {
    I r = idx;
    int64_t o0 = 0;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      I e = (I)sp.ext[d];
      I c = r % e;
      r /= e;
      o0 += (int64_t)c * sp.s0[d];
    }
    dst[o0] = 0.0;
  }
}

// Permuted add / copy whose destination and source are contiguous along different
// dimensions da and db: 32 x 32 tiles over (da, db) staged through shared memory, so
// reads run along the source's contiguous dimension and writes along the
// destination's; the other dimensions' offsets are decomposed once per tile.
template <bool COPY>
__global__ void __launch_bounds__(256) k_axpy_transpose(double* __restrict__ dst, const double* __restrict__ src,
                                                        Strided sp, int da, int db, int tiles_a, int tiles_b,
                                                        double alpha) {
  __shared__ double tile[32][33];
  int64_t blk = blockIdx.x;
  const int tbi = (int)(blk % tiles_b);
  blk /= tiles_b;
  const int tai = (int)(blk % tiles_a);
  int64_t rest = blk / tiles_a;
  int64_t o0 = 0, o1 = 0;
  for (int d = sp.ndim - 1; d >= 0; --d) {
    if (d == da || d == db) continue;
    const int64_t e = sp.ext[d], c = rest % e;
    rest /= e;
    o0 += c * sp.s0[d];
    o1 += c * sp.s1[d];
  }
  const int64_t ea = sp.ext[da], eb = sp.ext[db];
  const int64_t src_a = sp.s1[da], dst_b = sp.s0[db];
  const int a0 = tai * 32, b0 = tbi * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {  // read along b (source-contiguous)
    const int64_t a = a0 + i, b = b0 + threadIdx.x;
    if (a < ea && b < eb) tile[i][threadIdx.x] = src[o1 + a * src_a + b];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {  // write along a (destination-contiguous)
    const int64_t b = b0 + i, a = a0 + threadIdx.x;
    if (a < ea && b < eb) {
      const double v = tile[threadIdx.x][i];
      double* p = dst + o0 + a + b * dst_b;
      if (COPY)
        *p = v;
      else
        *p += alpha * v;
    }
  }
}

// The same when both are contiguous along one dimension d0: one block per row of the
// other dimensions (offsets decomposed once per row), threads along d0.
template <bool COPY>
__global__ void __launch_bounds__(256) k_axpy_rows(double* __restrict__ dst, const double* __restrict__ src,
                                                   Strided sp, int d0, int64_t rows, double alpha) {
  const int64_t ed = sp.ext[d0];
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t rest = row, o0 = 0, o1 = 0;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      if (d == d0) continue;
      const int64_t e = sp.ext[d], c = rest % e;
      rest /= e;
      o0 += c * sp.s0[d];
      o1 += c * sp.s1[d];
    }
    for (int64_t k = threadIdx.x; k < ed; k += blockDim.x) {
      if (COPY)
        dst[o0 + k] = src[o1 + k];
      else
        dst[o0 + k] += alpha * src[o1 + k];
    }
  }
}

// dispatch to the tiled kernels when the layouts allow; false: use the general one
template <bool COPY>
static bool launch_axpy_fast(double* dst, const double* src, const Strided& sp, double alpha, cudaStream_t st) {
  int da = -1, db = -1;
  for (int d = 0; d < sp.ndim; ++d) {
    if (sp.s0[d] == 1 && sp.ext[d] > 1) da = d;
    if (sp.s1[d] == 1 && sp.ext[d] > 1) db = d;
  }
  if (da < 0 || db < 0) return false;
  int64_t other = 1;
  for (int d = 0; d < sp.ndim; ++d)
    if (d != da && d != db) other *= sp.ext[d];
  if (da == db) {
    if (sp.ext[da] < 32) return false;
    const int threads = sp.ext[da] >= 256 ? 256 : (sp.ext[da] >= 128 ? 128 : 64);
    count_launches(1);
    k_axpy_rows<COPY><<<(int)std::min<int64_t>(other, 152 * 64), threads, 0, st>>>(dst, src, sp, da, other, alpha);
    return true;
  }
  if (sp.ext[da] < 8 || sp.ext[db] < 8) return false;
  const int ta = (int)((sp.ext[da] + 31) / 32), tb = (int)((sp.ext[db] + 31) / 32);
  const int64_t blocks = other * ta * tb;
  if (blocks > 0x7fffffffLL) return false;
  count_launches(1);
  k_axpy_transpose<COPY><<<(unsigned)blocks, dim3(32, 8), 0, st>>>(dst, src, sp, da, db, ta, tb, alpha);
  return true;
}

void launch_axpy_strided(double* dst, const double* src, const Strided& sp, double alpha, cudaStream_t st) {
  int64_t n = sp.total();
  if (n == 0) return;
  if (launch_axpy_fast<false>(dst, src, sp, alpha, st)) return;
  count_launches(1);
  if (n < (int64_t(1) << 31))
    k_axpy_strided<uint32_t, false><<<grid_for(n), 256, 0, st>>>(dst, src, sp, (uint32_t)n, alpha);
  else
    k_axpy_strided<uint64_t, false><<<grid_for(n), 256, 0, st>>>(dst, src, sp, (uint64_t)n, alpha);
}

void launch_copy_strided(double* dst, const double* src, const Strided& sp, cudaStream_t st) {
  int64_t n = sp.total();
  if (n == 0) return;
  if (launch_axpy_fast<true>(dst, src, sp, 1.0, st)) return;
  count_launches(1);
  if (n < (int64_t(1) << 31))
    k_axpy_strided<uint32_t, true><<<grid_for(n), 256, 0, st>>>(dst, src, sp, (uint32_t)n, 1.0);
  else
    k_axpy_strided<uint64_t, true><<<grid_for(n), 256, 0, st>>>(dst, src, sp, (uint64_t)n, 1.0);
}

void launch_zero_strided(double* dst, const Strided& sp, cudaStream_t st) {
  int64_t n = sp.total();
  if (n == 0) return;
  count_launches(1);
  if (n < (int64_t(1) << 31))
    k_zero_strided<uint32_t><<<grid_for(n), 256, 0, st>>>(dst, sp, (uint32_t)n);
  else
    k_zero_strided<uint64_t><<<grid_for(n), 256, 0, st>>>(dst, sp, (uint64_t)n);
}

// ---------------------------------------------------------------------------
// batched FP64 GEMM, 64x64 tiles, 16-deep k steps, 4x4 outputs per thread
// ---------------------------------------------------------------------------
constexpr int DT = 64, DK = 16;

// nsplit > 1: blockIdx.z = batch * nsplit + split; each split covers a K range and
// writes alpha * partial sum to part[split][b][m][n] (C is not touched).
__global__ void __launch_bounds__(256) k_dgemm(GemmArgs g, int nsplit, int kchunk, double* part) {
  __shared__ double As[DK][DT + 1];
  __shared__ double Bs[DK][DT + 1];
  const int b = blockIdx.z / nsplit;
  const int split = blockIdx.z % nsplit;
  const int kbeg = split * kchunk;
  const int kend = min(g.K, kbeg + kchunk);
  const int m0 = blockIdx.y * DT, n0 = blockIdx.x * DT;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const double* A = g.A + (int64_t)b * g.sAb;
  const double* B = g.B + (int64_t)b * g.sBb;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const bool akfast = (g.sAk == 1);
  const bool bkfast = (g.sBk == 1);
  for (int k0 = kbeg; k0 < kend; k0 += DK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + 256 * r;
      int kk, mm;
      if (akfast) {
        kk = e & 15;
        mm = e >> 4;
      } else {
        mm = e & 63;
        kk = e >> 6;
      }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < kend) ? A[(int64_t)m * g.sAm + (int64_t)k * g.sAk] : 0.0;
      int nn;
      if (bkfast) {
        kk = e & 15;
        nn = e >> 4;
      } else {
        nn = e & 63;
        kk = e >> 6;
      }
      int n = n0 + nn;
      k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < kend) ? B[(int64_t)n * g.sBn + (int64_t)k * g.sBk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (nsplit > 1) {
    double* P = part + ((int64_t)split * g.batch + b) * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int n = n0 + tx + 16 * j;
        if (n < g.N) P[(int64_t)m * g.N + n] = g.alpha * acc[i][j];
      }
    }
    return;
  }
  double* C = g.C + (int64_t)b * g.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double* c = C + (int64_t)m * g.sCm + (int64_t)n * g.sCn;
      double val = g.alpha * acc[i][j];
      if (g.beta != 0.0) val += g.beta * (*c);
      *c = val;
    }
  }
}

// Dot-product shapes (few outputs): one block per (split, output pair, batch).
// part[split][b][m][n] = alpha * sum_{k in split} A[b][m][k] B[b][n][k]
__global__ void __launch_bounds__(256) k_ddot_split(GemmArgs g, int nsplit, int64_t kchunk, double* part) {
  const int split = blockIdx.x;
  const int mn = blockIdx.y;
  const int b = blockIdx.z;
  const int m = mn / g.N, n = mn % g.N;
  const double* A = g.A + (int64_t)b * g.sAb + (int64_t)m * g.sAm;
  const double* B = g.B + (int64_t)b * g.sBb + (int64_t)n * g.sBn;
  const int64_t kbeg = split * kchunk;
  const int64_t kend = min((int64_t)g.K, kbeg + kchunk);
  double s = 0.0;
  for (int64_t k = kbeg + threadIdx.x; k < kend; k += blockDim.x) s = fma(A[k * g.sAk], B[k * g.sBk], s);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[((int64_t)split * g.batch + b) * g.M * g.N + mn] = g.alpha * sh[0];
}

// C = sum_split part + beta * C
__global__ void k_split_reduce(GemmArgs g, int nsplit, const double* __restrict__ part) {
  const int64_t tot = (int64_t)g.batch * g.M * g.N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = idx / ((int64_t)g.M * g.N);
    int64_t r = idx % ((int64_t)g.M * g.N);
    int64_t m = r / g.N, n = r % g.N;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * tot + idx];
    double* c = g.C + b * g.sCb + m * g.sCm + n * g.sCn;
    *c = (g.beta != 0.0) ? s + g.beta * (*c) : s;
  }
}

static void launch_dgemm_chunk(const GemmArgs& g, cudaStream_t st);

void launch_dgemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  if (g.K <= 0) throw std::runtime_error("dgemm: K must be positive");
  if (g.batch > 65535) throw std::runtime_error("dgemm: batch too large");
  // the M tiles index grid.y (<= 65535): split very tall products into row chunks
  const int64_t max_rows = (int64_t)65535 * DT;
  if (g.M > max_rows) {
    for (int64_t m0 = 0; m0 < g.M; m0 += max_rows) {
      GemmArgs c = g;
      c.M = (int)std::min<int64_t>(max_rows, g.M - m0);
      c.A = g.A + m0 * g.sAm;
      c.C = g.C + m0 * g.sCm;
      launch_dgemm_chunk(c, st);
    }
    return;
  }
  launch_dgemm_chunk(g, st);
}

// Matrix-vector shapes (N == 1): one warp per output row, lanes stride over K.
__global__ void __launch_bounds__(256) k_dgemv(GemmArgs g) {
  const int warps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)g.batch * g.M;
  for (int64_t r = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * warps) {
    const int64_t b = r / g.M, m = r % g.M;
    const double* A = g.A + b * g.sAb + m * g.sAm;
    const double* B = g.B + b * g.sBb;
    double s = 0.0;
    for (int64_t k = lane; k < g.K; k += 32) s = fma(A[k * g.sAk], B[k * g.sBk], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      double* c = g.C + b * g.sCb + m * g.sCm;
      *c = g.alpha * s + (g.beta != 0.0 ? g.beta * (*c) : 0.0);
    }
  }
}

// Rank-1 shapes (K == 1): C[b][m][n] = alpha A[b][m] B[b][n] + beta C.
__global__ void k_drank1(GemmArgs g) {
  const int64_t tot = (int64_t)g.batch * g.M * g.N;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = idx / ((int64_t)g.M * g.N);
    const int64_t r = idx % ((int64_t)g.M * g.N);
    const int64_t m = r / g.N, n = r % g.N;
    const double v = g.alpha * g.A[b * g.sAb + m * g.sAm] * g.B[b * g.sBb + n * g.sBn];
    double* c = g.C + b * g.sCb + m * g.sCm + n * g.sCn;
    *c = v + (g.beta != 0.0 ? g.beta * (*c) : 0.0);
  }
}

// Skinny shapes (N <= 16, the other extents large): C[b][m][n] = alpha sum_k A[b][m][k] B[b][n][k]
// + beta C for all n at once, so that A is read once (the 64 x 64 tiles would pad N to 64).
// The FP64 pipe bounds these (2 multiply-adds per clock per SM), so the kernel only has to keep
// it busy with coalesced loads of A.
//   ROWS = false: one 256-thread block per row m, the block's threads strided over k (A
//                 contiguous along k, or neither way), then a fixed-order block reduction;
//   ROWS = true:  32 rows per block, one per lane, the block's 8 warps strided over k (A
//                 contiguous along m: the warp's loads of A[m..m+31][k] coalesce, B[n][k] is
//                 the same for the warp), then a fixed-order reduction over the warps.
constexpr int SKINNY_N = 16;
template <bool ROWS>
__global__ void __launch_bounds__(256) k_dgemm_skinny(GemmArgs g) {
  const int N = g.N;
  if (!ROWS) {
    __shared__ double red[8][SKINNY_N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rows = (int64_t)g.batch * g.M;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
      const int64_t b = r / g.M, m = r % g.M;
      const double* A = g.A + b * g.sAb + m * g.sAm;
      const double* B = g.B + b * g.sBb;
      double acc[SKINNY_N];
#pragma unroll
      for (int n = 0; n < SKINNY_N; ++n) acc[n] = 0.0;
      for (int64_t k = threadIdx.x; k < g.K; k += blockDim.x) {
        const double a = A[k * g.sAk];
#pragma unroll
        for (int n = 0; n < SKINNY_N; ++n)
          if (n < N) acc[n] = fma(a, B[n * g.sBn + k * g.sBk], acc[n]);
      }
#pragma unroll
      for (int n = 0; n < SKINNY_N; ++n) {
        if (n >= N) break;
        double v = acc[n];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][n] = v;
      }
      __syncthreads();
      if (threadIdx.x < N) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        double* c = g.C + b * g.sCb + m * g.sCm + threadIdx.x * g.sCn;
        *c = g.alpha * v + (g.beta != 0.0 ? g.beta * (*c) : 0.0);
      }
      __syncthreads();
    }
  } else {
    // 32 rows per block (one per lane), the 8 warps strided over k, partial sums reduced in a
    // fixed order through shared memory
    __shared__ double red[8][SKINNY_N][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rows = (int64_t)g.batch * g.M;
    for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < rows; r0 += (int64_t)gridDim.x * 32) {
      const int64_t r = r0 + lane;
      double acc[SKINNY_N];
#pragma unroll
      for (int n = 0; n < SKINNY_N; ++n) acc[n] = 0.0;
      if (r < rows) {
        const int64_t b = r / g.M, m = r % g.M;
        const double* A = g.A + b * g.sAb + m * g.sAm;
        const double* B = g.B + b * g.sBb;
        for (int64_t k = warp; k < g.K; k += 8) {
          const double a = A[k * g.sAk];
#pragma unroll
          for (int n = 0; n < SKINNY_N; ++n)
            if (n < N) acc[n] = fma(a, B[n * g.sBn + k * g.sBk], acc[n]);
        }
      }
#pragma unroll
      for (int n = 0; n < SKINNY_N; ++n)
        if (n < N) red[warp][n][lane] = acc[n];
      __syncthreads();
      for (int q = threadIdx.x; q < N * 32; q += blockDim.x) {
        const int n = q >> 5, l = q & 31;
        const int64_t rr = r0 + l;
        if (rr < rows) {
          double v = 0.0;
#pragma unroll
          for (int w = 0; w < 8; ++w) v += red[w][n][l];
          const int64_t b = rr / g.M, m = rr % g.M;
          double* c = g.C + b * g.sCb + m * g.sCm + n * g.sCn;
          *c = g.alpha * v + (g.beta != 0.0 ? g.beta * (*c) : 0.0);
        }
      }
      __syncthreads();
    }
  }
}

static void launch_dgemm_chunk(const GemmArgs& g, cudaStream_t st) {
  if (g.K == 1) {
  count_launches(1);
    k_drank1<<<grid_for((int64_t)g.batch * g.M * g.N), 256, 0, st>>>(g);
    return;
  }
  if (g.N == 1 && (int64_t)g.M * g.batch >= 64) {
  count_launches(1);
    k_dgemv<<<grid_for((int64_t)g.batch * g.M * 32), 256, 0, st>>>(g);
    return;
  }
  if (g.M == 1 && (int64_t)g.N * g.batch >= 64) {
  count_launches(1);
    GemmArgs t = g;  // C^T = B A^T: swap the roles of A and B
    t.M = g.N;
    t.N = 1;
    t.A = g.B;
    t.sAb = g.sBb;
    t.sAm = g.sBn;
    t.sAk = g.sBk;
    t.B = g.A;
    t.sBb = g.sAb;
    t.sBn = g.sAm;
    t.sBk = g.sAk;
    t.sCm = g.sCn;
    t.sCn = g.sCm;
    k_dgemv<<<grid_for((int64_t)t.batch * t.M * 32), 256, 0, st>>>(t);
    return;
  }
  // skinny: N (or M, with the roles of A and B swapped) at most 16, enough rows to fill the
  // machine, K long enough that one pass over A dominates
  if (std::min(g.M, g.N) <= SKINNY_N && (int64_t)std::max(g.M, g.N) * g.batch >= 512 && g.K >= 32) {
    GemmArgs t = g;
    if (g.M < g.N) {  // C^T = B A^T
      t.M = g.N;
      t.N = g.M;
      t.A = g.B;
      t.sAb = g.sBb;
      t.sAm = g.sBn;
      t.sAk = g.sBk;
      t.B = g.A;
      t.sBb = g.sAb;
      t.sBn = g.sAm;
      t.sBk = g.sAk;
      t.sCm = g.sCn;
      t.sCn = g.sCm;
    }
    const int64_t rows = (int64_t)t.batch * t.M;
    count_launches(1);
    if (t.sAm == 1 && t.sAk != 1)
      k_dgemm_skinny<true><<<(int)std::min<int64_t>((rows + 31) / 32, 152 * 8), 256, 0, st>>>(t);
    else
      k_dgemm_skinny<false><<<(int)std::min<int64_t>(rows, 152 * 8), 256, 0, st>>>(t);
    return;
  }
  const int target = 2 * 152;
  const int64_t outputs = (int64_t)g.M * g.N;
  if (outputs <= 64 && g.batch <= 64 && g.K >= 4096) {
    int64_t nsplit = std::min<int64_t>(std::max<int64_t>(1, target / (outputs * g.batch)), (g.K + 2047) / 2048);
    nsplit = std::max<int64_t>(nsplit, 1);
    int64_t kchunk = (g.K + nsplit - 1) / nsplit;
    size_t bytes = (size_t)nsplit * g.batch * outputs * sizeof(double);
    double* part = (double*)dev_alloc(bytes, st, true);
    dim3 grid((unsigned)nsplit, (unsigned)outputs, g.batch);
    count_launches(2);
    k_ddot_split<<<grid, 256, 0, st>>>(g, (int)nsplit, kchunk, part);
    k_split_reduce<<<grid_for(g.batch * outputs), 256, 0, st>>>(g, (int)nsplit, part);
    dev_free(part, st, true);
    return;
  }
  const int64_t tm = (g.M + DT - 1) / DT, tn = (g.N + DT - 1) / DT;
  const int64_t tiles = tm * tn * g.batch;
  if (tm > 65535) throw std::runtime_error("dgemm: M too large");
  int nsplit = 1;
  if (tiles < target && g.K >= 8 * DK) {
    nsplit = (int)std::min<int64_t>(target / tiles, g.K / (4 * DK));
    nsplit = std::max(nsplit, 1);
    while ((int64_t)g.batch * nsplit > 65535) --nsplit;
  }
  if (nsplit == 1) {
  count_launches(1);
    dim3 grid((unsigned)tn, (unsigned)tm, g.batch);
    k_dgemm<<<grid, 256, 0, st>>>(g, 1, g.K, nullptr);
    return;
  }
  int kchunk = (g.K + nsplit - 1) / nsplit;
  kchunk = (kchunk + DK - 1) / DK * DK;
  nsplit = (g.K + kchunk - 1) / kchunk;
  size_t bytes = (size_t)nsplit * g.batch * g.M * g.N * sizeof(double);
  double* part = (double*)dev_alloc(bytes, st, true);
  dim3 grid((unsigned)tn, (unsigned)tm, (unsigned)(g.batch * nsplit));
  count_launches(2);
  k_dgemm<<<grid, 256, 0, st>>>(g, nsplit, kchunk, part);
  k_split_reduce<<<grid_for((int64_t)g.batch * g.M * g.N), 256, 0, st>>>(g, nsplit, part);
  dev_free(part, st, true);
}

// ---------------------------------------------------------------------------
// amplitude vectors
// ---------------------------------------------------------------------------
__device__ __forceinline__ double pair_weight(const VecShape& s, int64_t k) {
  // k indexes the whole vector; singles weigh 1
  int64_t n1 = s.n1();
  if (k < n1) return 1.0;
  uint32_t kd = (uint32_t)(k - n1);
  uint32_t v = (uint32_t)s.v, o = (uint32_t)s.o;
  uint32_t b = kd % v;
  kd /= v;
  uint32_t a = kd % v;
  kd /= v;
  uint32_t j = kd % o;
  uint32_t i = kd / o;
  return (i == j && a == b) ? 1.0 : 0.5;
}

// Packed inner products.  The pair weight is 1 on singles, 1/2 on doubles and 1 on
// the doubles diagonal (ai = bj), so <x|y> = sum_singles x y + 1/2 sum_doubles x y
// + 1/2 sum_diagonal x y: the partial kernel weighs by position only (no index
// arithmetic per element) and the final kernel adds the o*v diagonal terms.
constexpr int WD_BLOCK = 256;

template <int TP, int TQ>
__global__ void __launch_bounds__(WD_BLOCK) k_wdot_partial(VecShape s, const double* __restrict__ X, int64_t ldx,
                                                           int np, const double* __restrict__ Y, int64_t ldy, int nq,
                                                           double* __restrict__ work) {
  const int p0 = blockIdx.y * TP, q0 = blockIdx.z * TQ;
  const int pn = min(TP, np - p0), qn = min(TQ, nq - q0);
  double acc[TP][TQ];
#pragma unroll
  for (int p = 0; p < TP; ++p)
#pragma unroll
    for (int q = 0; q < TQ; ++q) acc[p][q] = 0.0;
  const int64_t dim = s.dim(), n1 = s.n1();
  const double* Xp[TP];
  const double* Yq[TQ];
#pragma unroll
  for (int p = 0; p < TP; ++p) Xp[p] = X + (int64_t)(p0 + min(p, pn - 1)) * ldx;
#pragma unroll
  for (int q = 0; q < TQ; ++q) Yq[q] = Y + (int64_t)(q0 + min(q, qn - 1)) * ldy;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim; k += (int64_t)gridDim.x * blockDim.x) {
    const double w = (k < n1) ? 1.0 : 0.5;
    double yv[TQ];
#pragma unroll
    for (int q = 0; q < TQ; ++q) yv[q] = w * Yq[q][k];
#pragma unroll
    for (int p = 0; p < TP; ++p) {
      const double xv = Xp[p][k];
#pragma unroll
      for (int q = 0; q < TQ; ++q) acc[p][q] = fma(xv, yv[q], acc[p][q]);
    }
  }
  __shared__ double red[WD_BLOCK / 32][TP * TQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < TP; ++p)
#pragma unroll
    for (int q = 0; q < TQ; ++q) {
      double v = acc[p][q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][p * TQ + q] = v;
    }
  __syncthreads();
  if (threadIdx.x < TP * TQ) {
    const int p = threadIdx.x / TQ, q = threadIdx.x % TQ;
    if (p < pn && q < qn) {
      double t = 0.0;
      for (int w2 = 0; w2 < WD_BLOCK / 32; ++w2) t += red[w2][threadIdx.x];
      work[((int64_t)blockIdx.x * np + (p0 + p)) * nq + (q0 + q)] = t;
    }
  }
}

// G[p][q] = sum over chunks + 1/2 sum over the doubles diagonal x_iiaa y_iiaa
__global__ void k_wdot_final(VecShape s, int nchunks, int np, int nq, const double* __restrict__ work,
                             const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y, int64_t ldy,
                             double* G, int ldg) {
  const int pq = blockIdx.x;
  const int p = pq / nq, q = pq % nq;
  double sum = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) sum += work[((int64_t)c * np + p) * nq + q];
  const int64_t n1 = s.n1();
  const int o = s.o, v = s.v;
  const double* x = X + (int64_t)p * ldx + n1;
  const double* y = Y + (int64_t)q * ldy + n1;
  for (int ia = threadIdx.x; ia < o * v; ia += blockDim.x) {
    const int i = ia / v, a = ia % v;
    const int64_t e = (((int64_t)i * o + i) * v + a) * v + a;
    sum = fma(0.5 * x[e], y[e], sum);
  }
  __shared__ double sh[128];
  sh[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 64; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) G[p * ldg + q] = sh[0];
}

static int wdot_chunks() { return 152 * 2; }

int64_t wdot_work_size(int np, int nq) { return (int64_t)wdot_chunks() * np * nq; }

void launch_wdot(const VecShape& s, const double* X, int64_t ldx, int np, const double* Y, int64_t ldy, int nq,
                 double* G, int ldg, double* work, cudaStream_t st) {
  if (np <= 0 || nq <= 0) return;
  const int nch = wdot_chunks();
  count_launches(2);
  if (np == 1 && nq == 1) {
    k_wdot_partial<1, 1><<<dim3(nch, 1, 1), WD_BLOCK, 0, st>>>(s, X, ldx, np, Y, ldy, nq, work);
  } else if (nq == 1) {
    k_wdot_partial<4, 1><<<dim3(nch, (np + 3) / 4, 1), WD_BLOCK, 0, st>>>(s, X, ldx, np, Y, ldy, nq, work);
  } else if (np == 1) {
    k_wdot_partial<1, 4><<<dim3(nch, 1, (nq + 3) / 4), WD_BLOCK, 0, st>>>(s, X, ldx, np, Y, ldy, nq, work);
  } else {
    k_wdot_partial<4, 4><<<dim3(nch, (np + 3) / 4, (nq + 3) / 4), WD_BLOCK, 0, st>>>(s, X, ldx, np, Y, ldy, nq,
                                                                                    work);
  }
  k_wdot_final<<<np * nq, 128, 0, st>>>(s, nch, np, nq, work, X, ldx, Y, ldy, G, ldg);
}

__global__ void k_lincomb(int64_t dim, const double* __restrict__ X, int64_t ldx, int np, const double* __restrict__ c,
                          int ldc, double* __restrict__ Y, int64_t ldy, int nq, bool accumulate) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim; k += (int64_t)gridDim.x * blockDim.x) {
    for (int q0 = 0; q0 < nq; q0 += 8) {
      double acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0;
      for (int p = 0; p < np; ++p) {
        double xv = X[(int64_t)p * ldx + k];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q0 + q < nq) acc[q] = fma(c[p * ldc + q0 + q], xv, acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q0 + q >= nq) break;
        double* y = Y + (int64_t)(q0 + q) * ldy + k;
        *y = accumulate ? (*y + acc[q]) : acc[q];
      }
    }
  }
}

// The same combination in double-float arithmetic on the FP32 pipe, which issues 64 times as
// many operations per clock as the FP64 pipe on this chip (k_lincomb is FP64-bound: nq
// multiply-adds per loaded element).  Each X element is cut into two floats from its bits
// (double_to_float2), each coefficient into two floats once per block; a term c x is
// ch xh (its rounding error recovered exactly by an FMA) plus ch xl + cl xh, and the sum is
// carried as an unevaluated float pair (two-sum with explicit round-to-nearest operations, so
// that no multiply-add is contracted into it).  Accuracy about 2^-44 of sum_p |c_pq X_p[k]|,
// against 2^-53 for FP64.  Used for the Ritz vectors of the Davidson solver (fp64grade): their
// coefficients are eigenvector components of an orthonormal basis, so the error stays 2^-44 of
// the vector.  Combinations whose coefficients can cancel strongly (DIIS extrapolation, GMRES
// updates, orthogonalisation of a nearly dependent vector) keep k_lincomb.
__global__ void __launch_bounds__(256) k_lincomb_df(int64_t dim, const double* __restrict__ X, int64_t ldx, int np,
                                                    const double* __restrict__ c, int ldc, double* __restrict__ Y,
                                                    int64_t ldy, int nq, bool accumulate) {
  extern __shared__ float2 cs[];  // [np][nq]: (high, low) floats of each coefficient
  for (int i = threadIdx.x; i < np * nq; i += blockDim.x) {
    const int p = i / nq, q = i % nq;
    const double v = c[p * ldc + q];
    const float h = __double2float_rn(v);
    cs[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim; k += (int64_t)gridDim.x * blockDim.x) {
    for (int q0 = 0; q0 < nq; q0 += 8) {
      float sh[8], sl[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q] = sl[q] = 0.0f;
#pragma unroll 4
      for (int p = 0; p < np; ++p) {
        float xh, xl;
        double_to_float2(X[(int64_t)p * ldx + k], xh, xl);
        const float2* cp = cs + p * nq + q0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q0 + q < nq) {
            const float2 cc = cp[q];
            const float ph = __fmul_rn(cc.x, xh);
            const float pe = __fmaf_rn(cc.x, xh, -ph);  // ch xh - ph, exact
            const float lo = __fmaf_rn(cc.x, xl, __fmaf_rn(cc.y, xh, pe));
            const float t = __fadd_rn(sh[q], ph);
            const float bp = __fsub_rn(t, sh[q]);
            const float err = __fadd_rn(__fsub_rn(sh[q], __fsub_rn(t, bp)), __fsub_rn(ph, bp));
            sh[q] = t;
            sl[q] = __fadd_rn(sl[q], __fadd_rn(err, lo));
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q0 + q >= nq) break;
        const double v = (double)sh[q] + (double)sl[q];
        double* y = Y + (int64_t)(q0 + q) * ldy + k;
        *y = accumulate ? (*y + v) : v;
      }
    }
  }
}

void launch_lincomb(const VecShape& s, const double* X, int64_t ldx, int np, const double* c, int ldc, double* Y,
                    int64_t ldy, int nq, bool accumulate, cudaStream_t st, bool fp64grade) {
  count_launches(1);
  int64_t dim = s.dim();
  const size_t smem = (size_t)np * nq * sizeof(float2);
  if (fp64grade && smem <= 32 * 1024)
    k_lincomb_df<<<grid_for(dim), 256, smem, st>>>(dim, X, ldx, np, c, ldc, Y, ldy, nq, accumulate);
  else
    k_lincomb<<<grid_for(dim), 256, 0, st>>>(dim, X, ldx, np, c, ldc, Y, ldy, nq, accumulate);
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = a * x[k] + (b == 0.0 ? 0.0 : b * y[k]);
}

void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  if (n > 0) {
    count_launches(1);
    k_axpby<<<grid_for(n), 256, 0, st>>>(n, a, x, b, y);
  }
}

__global__ void k_precond(VecShape s, const double* __restrict__ eps, const double* __restrict__ x,
                          double* __restrict__ y, double shift) {
  const int64_t dim = s.dim(), n1 = s.n1();
  const uint32_t o = s.o, v = s.v;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim; k += (int64_t)gridDim.x * blockDim.x) {
    double d;
    if (k < n1) {
      uint32_t a = (uint32_t)k % v, i = (uint32_t)k / v;
      d = eps[o + a] - eps[i];
    } else {
      uint32_t kd = (uint32_t)(k - n1);
      uint32_t b = kd % v;
      kd /= v;
      uint32_t a = kd % v;
      kd /= v;
      uint32_t j = kd % o, i = kd / o;
      d = eps[o + a] + eps[o + b] - eps[i] - eps[j];
    }
    y[k] = x[k] / (d - shift);
  }
}

void launch_precond(const VecShape& s, const double* eps, const double* x, double* y, double shift,
                    cudaStream_t st) {
  k_precond<<<grid_for(s.dim()), 256, 0, st>>>(s, eps, x, y, shift);
  count_launches(1);
}

__global__ void k_weight(VecShape s, const double* __restrict__ x, double* __restrict__ y, int nvec, int64_t ld) {
  const int64_t dim = s.dim();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim * nvec;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t vi = k / dim, e = k % dim;
    y[vi * ld + e] = pair_weight(s, e) * x[vi * ld + e];
  }
}

void launch_weight(const VecShape& s, const double* x, double* y, int nvec, int64_t ld, cudaStream_t st) {
  count_launches(1);
  k_weight<<<grid_for(s.dim() * nvec), 256, 0, st>>>(s, x, y, nvec, ld);
}

__global__ void k_packed_grad(VecShape s, const double* __restrict__ g, double* __restrict__ y, int nvec,
                              int64_t ld) {
  const int64_t dim = s.dim(), n1 = s.n1();
  const uint32_t o = s.o, v = s.v;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < dim * nvec;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t vi = k / dim, e = k % dim;
    const double* gv = g + vi * ld;
    double r;
    if (e < n1) {
      r = gv[e];
    } else {
      uint32_t kd = (uint32_t)(e - n1);
      uint32_t b = kd % v;
      uint32_t t = kd / v;
      uint32_t a = t % v;
      t /= v;
      uint32_t j = t % o, i = t / o;
      if (i == j && a == b) {
        r = gv[e];
      } else {
        int64_t tr = n1 + (((int64_t)j * o + i) * v + b) * v + a;
        r = gv[e] + gv[tr];
      }
    }
    y[vi * ld + e] = r;
  }
}

void launch_packed_grad(const VecShape& s, const double* g, double* y, int nvec, int64_t ld, cudaStream_t st) {
  if (g == y) throw std::runtime_error("packed_grad must be out of place");
  count_launches(1);
  k_packed_grad<<<grid_for(s.dim() * nvec), 256, 0, st>>>(s, g, y, nvec, ld);
}

__global__ void k_maxabs_partial(int64_t n, const double* __restrict__ x, double* work, int with_index) {
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double a = fabs(x[k]);
    if (a > best) {
      best = a;
      bi = k;
    }
  }
  __shared__ double sb[256];
  __shared__ int64_t si[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      double ob = sb[threadIdx.x + off];
      int64_t oi = si[threadIdx.x + off];
      if (ob > sb[threadIdx.x] || (ob == sb[threadIdx.x] && oi < si[threadIdx.x])) {
        sb[threadIdx.x] = ob;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    work[2 * blockIdx.x] = sb[0];
    work[2 * blockIdx.x + 1] = (double)si[0];
  }
}

__global__ void k_maxabs_final(int nb, const double* work, const double* x, double* out, int with_index) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double best = -1.0, bi = 0.0;
  for (int b = 0; b < nb; ++b) {
    double v = work[2 * b], i = work[2 * b + 1];
    if (v > best || (v == best && i < bi)) {
      best = v;
      bi = i;
    }
  }
  if (with_index) {
    out[0] = bi;
    out[1] = x[(int64_t)bi];
  } else {
    out[0] = best;
  }
}

void launch_maxabs(int64_t n, const double* x, double* out, double* work, cudaStream_t st) {
  int nb = 256;
  count_launches(2);
  k_maxabs_partial<<<nb, 256, 0, st>>>(n, x, work, 0);
  k_maxabs_final<<<1, 32, 0, st>>>(nb, work, x, out, 0);
}

void launch_argmaxabs(int64_t n, const double* x, double* out, double* work, cudaStream_t st) {
  int nb = 256;
  count_launches(2);
  k_maxabs_partial<<<nb, 256, 0, st>>>(n, x, work, 1);
  k_maxabs_final<<<1, 32, 0, st>>>(nb, work, x, out, 1);
}

__global__ void k_dot_partial(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* work) {
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[k], y[k], s);
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) work[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(int nb, const double* work, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += work[b];
  out[0] = s;
}

// partial sums of the biorthonormal-bra metric of a vector a (singles [i][a], doubles
// [i][j][a][b] pair-symmetric): 1/2 a_ia^2 and (2 A_ijab^2 + A_ijab A_ijba)/12, plus
// 3/4 A_iiaa^2 on the diagonal ai = bj
__global__ void k_bra_metric_partial(VecShape vs, const double* __restrict__ a, double* work) {
  const int o = vs.o, v = vs.v;
  const int64_t n1 = vs.n1(), n = vs.dim();
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[k];
    if (k < n1) {
      s = fma(0.5 * x, x, s);
      continue;
    }
    const int64_t e = k - n1;
    const int b = (int)(e % v);
    int64_t r = e / v;
    const int aa = (int)(r % v);
    r /= v;
    const int j = (int)(r % o), i = (int)(r / o);
    const double xs = a[n1 + (((int64_t)i * o + j) * v + b) * v + aa];
    s += (2.0 * x * x + x * xs) * (1.0 / 12.0);
    if (i == j && aa == b) s += 0.75 * x * x;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) work[blockIdx.x] = sh[0];
}

// x2[i][j][a][b] = t2[i][j][a][b] - t1[i][a] t1[j][b] (the doubles of exp(-T)'s coefficients, negated)
__global__ void k_t2_minus_t1t1(VecShape vs, const double* __restrict__ t, double* __restrict__ x) {
  const int o = vs.o, v = vs.v;
  const int64_t n1 = vs.n1(), n2 = vs.dim() - n1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % v);
    int64_t r = e / v;
    const int aa = (int)(r % v);
    r /= v;
    const int j = (int)(r % o), i = (int)(r / o);
    x[n1 + e] = t[n1 + e] - t[(int64_t)i * v + aa] * t[(int64_t)j * v + b];
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n1; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = t[e];
}

void launch_bra_metric(const VecShape& s, const double* a, double* out, double* work, cudaStream_t st) {
  const int nb = 512;
  count_launches(2);
  k_bra_metric_partial<<<nb, 256, 0, st>>>(s, a, work);
  k_sum_final<<<1, 32, 0, st>>>(nb, work, out);
}

void launch_t2_minus_t1t1(const VecShape& s, const double* t, double* x, cudaStream_t st) {
  count_launches(1);
  k_t2_minus_t1t1<<<(int)std::min<int64_t>((s.dim() + 255) / 256, 152 * 16), 256, 0, st>>>(s, t, x);
}

void launch_dot(int64_t n, const double* x, const double* y, double* out, double* work, cudaStream_t st) {
  int nb = 512;
  count_launches(2);
  k_dot_partial<<<nb, 256, 0, st>>>(n, x, y, work);
  k_sum_final<<<1, 32, 0, st>>>(nb, work, out);
}

// <L|tau_sigma|(r0 + R)>: singles y[j,b] = r0 L1[j,b] + sum_ia (1 + delta_ia,jb) L2[i,j,a,b] R1[i,a];
// doubles y2 = r0 L2.  (A single tau_jb on R1 gives a double; only <L2| sees it.)
__global__ void k_tau_singles(VecShape s, double r0, const double* __restrict__ L, const double* __restrict__ R,
                              double* __restrict__ y) {
  const int o = s.o, v = s.v;
  const int jb = blockIdx.x;
  const int j = jb / v, b = jb % v;
  const int64_t n1 = s.n1();
  const double* L2 = L + n1;
  double acc = 0.0;
  for (int ia = threadIdx.x; ia < o * v; ia += blockDim.x) {
    int i = ia / v, a = ia % v;
    double l = L2[(((int64_t)i * o + j) * v + a) * v + b];
    double f = (i == j && a == b) ? 2.0 : 1.0;
    acc = fma(f * l, R[ia], acc);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) y[jb] = r0 * L[jb] + sh[0];
}

void launch_tau_expectation(const VecShape& s, double r0, const double* L, const double* R, double* y,
                            cudaStream_t st) {
  count_launches(2);
  k_tau_singles<<<s.o * s.v, 256, 0, st>>>(s, r0, L, R, y);
  int64_t n2 = s.dim() - s.n1();
  k_axpby<<<grid_for(n2), 256, 0, st>>>(n2, r0, L + s.n1(), 0.0, y + s.n1());
}

}  // namespace ccsd

namespace ccsd {
namespace {
// block-wide sum of one value per thread (blockDim.x a multiple of 32, at most 1024)
__device__ double block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = x;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__global__ void k_branching_plane(int n, double gap, const double* __restrict__ gk, const double* __restrict__ gl,
                                  const double* __restrict__ f, double* __restrict__ out) {
  __shared__ double red[32];
  double* g = out;
  double* h = out + n;
  double* G = out + 2 * n;
  double gg = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double gi = gl[i] - gk[i];
    g[i] = gi;
    h[i] = gap * f[i];
    gg += gi * gi;
  }
  const double gnorm = sqrt(block_sum(gg, red));
  const double inv_g = gnorm > 0.0 ? 1.0 / gnorm : 0.0;
  // h with its component along q1 = g/|g| removed
  double hq = 0.0, hh = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    hq += h[i] * g[i] * inv_g;
    hh += h[i] * h[i];
  }
  hq = block_sum(hq, red);
  const double hnorm = sqrt(block_sum(hh, red));
  double pp = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double hp = h[i] - hq * g[i] * inv_g;
    pp += hp * hp;
  }
  const double pnorm = sqrt(block_sum(pp, red));
  const bool two = pnorm > 1e-12 * fmax(hnorm, 1e-300);
  const double inv_p = two ? 1.0 / pnorm : 0.0;
  // projections of gl on q1 and q2
  double a1 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double q1 = g[i] * inv_g;
    const double q2 = (h[i] - hq * q1) * inv_p;
    a1 += gl[i] * q1;
    a2 += gl[i] * q2;
  }
  a1 = block_sum(a1, red);
  a2 = block_sum(a2, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double q1 = g[i] * inv_g;
    const double q2 = (h[i] - hq * q1) * inv_p;
    G[i] = gl[i] - a1 * q1 - a2 * q2 + 2.0 * gap * q1;
  }
}
}  // namespace

__global__ void k_antisymmetric_part(int n, const double* __restrict__ D, double* __restrict__ out) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = x / n, q = x % n;
    out[x] = 0.5 * (D[x] - D[q * n + p]);
  }
}

void launch_antisymmetric_part(int n, const double* D, double* out, cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  count_launches(1);
  k_antisymmetric_part<<<(int)std::min<int64_t>((nn + 255) / 256, 152 * 8), 256, 0, st>>>(n, D, out);
}

void launch_branching_plane(int n, double gap, const double* gk, const double* gl, const double* f, double* out,
                            cudaStream_t st) {
  count_launches(1);
  k_branching_plane<<<1, 256, 0, st>>>(n, gap, gk, gl, f, out);
}
}  // namespace ccsd
