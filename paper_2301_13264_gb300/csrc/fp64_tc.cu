// FP64-grade contraction on the tensor cores, for the FP64 residuals of the
// refined mixed-precision solves.  The operand splitting follows the error-free
// transformation of matrix products of Ozaki, Ogita, Oishi and Rump (Numer.
// Algorithms 59, 2012: fixed-point slices whose partial products are exact),
// adapted here to bf16 operands with FP32 TMEM accumulation: exactness comes from
// bounding each accumulator's sum per K chunk, not from integer arithmetic.
//
// Operand layout.  An FP64 operand X (rows x K) is scaled row by row by 2^-e_r,
// with e_r the smallest exponent such that every |X_rk| < 2^e_r, and cut into
// S = 7 fixed-point slices of 7 bits:
//     X_rk 2^-e_r = 2^-6 (a_0 + a_1 + ... + a_6) + rest,   a_s = q_s 2^-7s,
// q_0 = round(64 x) and q_s = round(128 r_s) of the remainder r_s, so every q_s
// is an integer in [-64, 64] and every a_s is exact in bf16; |rest| <= 2^-49.
// The slices live in [S][rows_p][Kp] bf16 planes (zero padding), followed by
// the rows_p int exponents.
//
// Arithmetic.  A product a_s b_t is an integer times 2^-7(s+t) of magnitude at
// most 2^12 2^-7(s+t).  The products of one level l = s + t (l + 1 <= 7 pairs)
// summed over a K chunk of 512 stay within 7 * 512 * 2^12 < 2^24 units of
// 2^-7l, so their FP32 sum in TMEM is exact whatever the order of additions.
// Each of the levels 0..6 has its own TMEM accumulator (128 x 64 FP32 columns);
// after every chunk the read-out warps convert them to integers in units of
// 2^-35 (exact for levels 0..5, level 6 rounded) and add them into one 64-bit
// integer per output element, so the sum over K is exact up to that rounding
// (2^-47 of the largest product per chunk).  A chunk adds at most 2^56.1 units,
// so a split covers at most 56 chunks (K <= 28672).  Products with s + t >= 7 are
// dropped.  The output is
//     C_mn = alpha 2^(e_m + f_n - 47) acc_mn + beta C_mn,
// with an error per K term of about 2^-46 max_k |A_mk| max_k |B_nk| (the dropped
// levels and the slice remainders, of either sign) and one final rounding.
//
// Kernel.  One 128 x 64 output tile per CTA, 10 warps, 1 CTA per SM (177 KB of
// shared memory, all 512 TMEM columns).  Warp 0 lane 0 loads, per 64-wide K tile,
// the 7 slices of the B tile into one of 2 B-group buffers and the A slices one by
// one into a 4-stage ring (TMA, 3-D maps whose third coordinate is the slice);
// warp 1 lane 0 issues, for each A slice s, the products with B slices t <= 6 - s
// into the level-(s+t) accumulators (tcgen05.mma kind::f16, 128 x 64nt x 16: up to four
// B slices, adjacent in shared memory, against adjacent level accumulators), and
// after the last K tile of a chunk commits to the read-out barrier; warps 2..9
// (TMEM lane quarter = warp mod 4, one half of the columns each) read the seven
// accumulators, release them to the MMA warp and, after the last chunk, write
// the FP64 tile through shared memory.  Split-K over
// blockIdx.z writes FP64 partial tiles that a second kernel sums.  Every wait is
// bounded; on timeout the kernel raises the error flag, drains its own copies and
// MMAs (bounded), frees TMEM and exits.
#include "alloc.h"
#include "fp64_tc.h"

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <stdexcept>
#include <string>

#include "tcgen05.cuh"

namespace ccsd {
namespace oz {

using tc::BK;
using tc::BM;

constexpr int A_BYTES = BM * BK * 2;    // one A slice tile, 16 KB
constexpr int B_BYTES = BN * BK * 2;    // one B slice tile, 8 KB
constexpr int BG_BYTES = S * B_BYTES;   // the 7 B slice tiles of one K tile, 56 KB
constexpr int A_STAGES = 4, B_STAGES = 2;
constexpr int NTHREADS = 320;  // 2 control warps + 8 read-out warps
constexpr int HALF = BN / 2;      // columns per read-out warp
constexpr int SMEM_BYTES = B_STAGES * BG_BYTES + A_STAGES * A_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;     // 7 level accumulators of BN columns
static_assert(S * BN <= (int)TMEM_COLS, "level accumulators exceed TMEM");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

struct Params {
  int M, N;
  int kt_total;      // 64-wide K tiles
  int kt_per_split;  // K tiles per blockIdx.z
  const int* ea;     // row exponents of A and B
  const int* eb;
  double* C;
  long long sCm, sCn;
  double* part;      // split-K partial tiles [z][M][N]
  double alpha;
  int beta_zero;
  int* err;
  int ostr;
  Strided om, on;
  long long budget;  // clock cycles a pipeline wait may take before the kernel gives up
  int mt, nt, group_m;  // output tiles (rows, columns) and rows per raster group (tc::raster_tile)
};

__device__ __forceinline__ long long dim_off(long long x, const Strided& g) {
  long long off = 0;
  for (int d = g.ndim - 1; d >= 0; --d) {
    const long long e = g.ext[d];
    off += (x % e) * g.s0[d];
    x /= e;
  }
  return off;
}

// kind::f16 instruction descriptor (FP32 accumulator, bf16 A and B, K-major) for M = 128 and
// N = n (a multiple of 16 up to 256)
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Wait bounded by time only (used before freeing TMEM, when the error flag may be up).
__device__ __forceinline__ bool wait_quiet(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(bar, parity))
    if (clock64() - t0 > tc::TIMEOUT_CYCLES) return false;
  return true;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Add the seven levels' chunk sums (TMEM columns L*BN + ..) into the integer accumulators,
// in units of 2^-35: level L holds an integer times 2^-7L below 2^24 units, so for L <= 5 the
// scaled value 2^7L V and its conversion are exact; level 6 is rounded to 2^-35.
__device__ __forceinline__ void read_levels(uint32_t taddr, long long (&acc)[HALF]) {
#pragma unroll 1
  for (int L = 0; L < S; ++L) {
    const int sh = min(7 * L, 35);
    const float fs = (float)(1LL << sh);
    const long long mul = 1LL << (35 - sh);
#pragma unroll
    for (int c = 0; c < HALF; c += 16) {
      uint32_t r[16];
      tmem_ld16(taddr + (uint32_t)(L * BN + c), r);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        acc[c + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * fs) * mul;
    }
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_dgemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, Params p) {
  extern __shared__ uint8_t smem_raw[];
  volatile int* err = p.err;
  if (*err) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = smem;
  uint8_t* sA = smem + B_STAGES * BG_BYTES;
  uint64_t* bars = (uint64_t*)(sA + A_STAGES * A_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 16);
  const uint32_t bfull = tc::smem_u32(bars), bempty = tc::smem_u32(bars + 2);
  const uint32_t afull = tc::smem_u32(bars + 4), aempty = tc::smem_u32(bars + 8);
  const uint32_t accfull = tc::smem_u32(bars + 12), accempty = tc::smem_u32(bars + 13);
  const uint32_t done = tc::smem_u32(bars + 14);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm, tn;
  tc::raster_tile(blockIdx.x, p.mt, p.nt, p.group_m, tm, tn);
  const int m0 = tm * BM, n0 = tn * BN;
  const int kt0 = blockIdx.z * p.kt_per_split;
  const int nkt = max(0, min(p.kt_total, kt0 + p.kt_per_split) - kt0);
  const int nch = (nkt + KC_TILES - 1) / KC_TILES;

  if (threadIdx.x == 0) {
    for (int i = 0; i < B_STAGES; ++i) {
      tc::mbar_init(bfull + 8 * i, 1);
      tc::mbar_init(bempty + 8 * i, 1);
    }
    for (int i = 0; i < A_STAGES; ++i) {
      tc::mbar_init(afull + 8 * i, 1);
      tc::mbar_init(aempty + 8 * i, 1);
    }
    tc::mbar_init(accfull, 1);
    tc::mbar_init(accempty, 8);
    tc::mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sA0 = tc::smem_u32(sA), sB0 = tc::smem_u32(sB);

  if (warp == 0) {
    if (lane == 0) {
      // producer
      int nb = 0, na = 0;
      bool ok = true;
      for (int k = 0; k < nkt && ok; ++k) {
        const int bs = k % B_STAGES;
        if (!tc::mbar_wait(bempty + 8 * bs, ((uint32_t)(k / B_STAGES) & 1u) ^ 1u, err, p.budget)) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(bfull + 8 * bs, BG_BYTES);
        for (int t = 0; t < S; ++t)
          tc::tma_load_3d(sB0 + bs * BG_BYTES + t * B_BYTES, &tb, bfull + 8 * bs, (kt0 + k) * BK, n0, t);
        ++nb;
        for (int s = 0; s < S; ++s) {
          const int as = na % A_STAGES;
          if (!tc::mbar_wait(aempty + 8 * as, ((uint32_t)(na / A_STAGES) & 1u) ^ 1u, err, p.budget)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(afull + 8 * as, A_BYTES);
          tc::tma_load_3d(sA0 + as * A_BYTES, &ta, afull + 8 * as, (kt0 + k) * BK, m0, s);
          ++na;
        }
      }
      if (!ok) {
        atomicExch((int*)p.err, 1);
        // wait (bounded) for this CTA's copies still in flight
        for (int i = nb - 1; i >= 0 && i >= nb - B_STAGES; --i)
          wait_quiet(bfull + 8 * (i % B_STAGES), (uint32_t)(i / B_STAGES) & 1u);
        for (int i = na - 1; i >= 0 && i >= na - A_STAGES; --i)
          wait_quiet(afull + 8 * (i % A_STAGES), (uint32_t)(i / A_STAGES) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issue
      int na = 0;
      bool ok = true;
      for (int k = 0; k < nkt && ok; ++k) {
        const int kc = k % KC_TILES, ch = k / KC_TILES;
        if (kc == 0 && ch > 0) {
          // the previous chunk's accumulators must have been read out
          if (!tc::mbar_wait(accempty, (uint32_t)(ch - 1) & 1u, err, p.budget)) {
            ok = false;
            break;
          }
          tc::fence_after();
        }
        const int bs = k % B_STAGES;
        if (!tc::mbar_wait(bfull + 8 * bs, (uint32_t)(k / B_STAGES) & 1u, err, p.budget)) {
          ok = false;
          break;
        }
        tc::fence_after();
        for (int s = 0; s < S; ++s) {
          const int as = na % A_STAGES;
          if (!tc::mbar_wait(afull + 8 * as, (uint32_t)(na / A_STAGES) & 1u, err, p.budget)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t a0 = sA0 + as * A_BYTES;
          // The products a_s b_t, t = 0 .. 6-s, land in the levels s .. 6, whose accumulators are
          // contiguous in TMEM, and the B slices t are contiguous 64-row tiles in the B group: up
          // to four of them form one B operand of N = 64 nt rows, so one MMA covers nt products.
          for (int t0 = 0; t0 < S - s; t0 += 4) {
            const int nt = min(4, S - s - t0);
            const uint32_t b0 = sB0 + bs * BG_BYTES + t0 * B_BYTES;
            const uint32_t d = tmem + (uint32_t)((s + t0) * BN);
            const uint32_t idsc = idesc_n(BN * nt);
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)
              tc::mma_bf16(d, tc::smem_desc(a0 + 32 * j), tc::smem_desc(b0 + 32 * j), idsc,
                           (kc == 0 && s == 0 && j == 0) ? 0u : 1u);
          }
          tc::mma_commit(aempty + 8 * as);
          ++na;
        }
        if (!ok) break;
        tc::mma_commit(bempty + 8 * bs);
        if (kc == KC_TILES - 1 || k == nkt - 1) tc::mma_commit(accfull);
      }
      if (!ok) atomicExch((int*)p.err, 1);
      tc::mma_commit(done);  // fires once every issued MMA has completed
    }
    __syncwarp();
  } else {
    // read-out warps 2..9: TMEM lane quarter q, columns h*32 .. h*32+31 of every level
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = m0 + q * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * HALF);
    long long acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0;
    bool ok = true;
    for (int ch = 0; ch < nch; ++ch) {
      if (!tc::mbar_wait(accfull, (uint32_t)ch & 1u, err, p.budget)) {
        ok = false;
        break;
      }
      tc::fence_after();
      read_levels(taddr, acc);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty);
    }
    if (!ok) atomicExch((int*)p.err, 1);
    const bool split = (gridDim.z > 1);
    const bool ostr = !split && p.ostr;
    // Every MMA and every copy has completed (last read-out barrier): the stage
    // buffers are idle.  The tile goes through shared memory (B buffers: [128][65]
    // doubles) so that the global writes are row-contiguous across threads.
    double* stage = reinterpret_cast<double*>(sB);
    long long* coloff = reinterpret_cast<long long*>(sA);
    long long* rowoff = coloff + BN;
    const int tid = threadIdx.x - 64;
    if (ok) {
      const int r = q * 32 + lane;
      const int em = (row < p.M) ? p.ea[row] : 0;
      const double sm = ldexp(p.alpha, em - 47);
#pragma unroll
      for (int j = 0; j < HALF; ++j) {
        const int en = p.eb[n0 + h * HALF + j];  // padding rows of B carry exponent 0
        double v;
        if (em == NONFINITE || en == NONFINITE) {
          v = __longlong_as_double(0x7ff8000000000000LL);
        } else {
          // 2^en from its bit pattern in the normal range
          const double pn =
              (en > -1000 && en < 1000) ? __longlong_as_double((long long)(en + 1023) << 52) : ldexp(1.0, en);
          v = (double)acc[j] * (sm * pn);
        }
        stage[r * (BN + 1) + h * HALF + j] = v;
      }
      if (ostr) {
        if (tid < BN) coloff[tid] = (n0 + tid < p.N) ? dim_off(n0 + tid, p.on) : 0;
        if (tid < BM) rowoff[tid] = (m0 + tid < p.M) ? dim_off(m0 + tid, p.om) : 0;
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (ok && !*err) {
      const long long cs = split ? 1 : p.sCn;
      for (int idx = tid; idx < BM * BN; idx += 256) {
        const int r = idx / BN, c = idx % BN;
        const int m = m0 + r, n = n0 + c;
        if (m < p.M && n < p.N) {
          const double v = stage[r * (BN + 1) + c];
          double* dst = split ? p.part + ((long long)blockIdx.z * p.M + m) * p.N + n
                              : (ostr ? p.C + rowoff[r] + coloff[c] : p.C + (long long)m * p.sCm + (long long)n * cs);
          *dst = (split || p.beta_zero) ? v : (*dst + v);
        }
      }
    }
  }

  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) {
    if (!wait_quiet(done, 0)) atomicExch((int*)p.err, 1);
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// offsets of a strided gather over dims [d0, d1): off[x] = sum_d coord_d(x) * g.s1[d]
__global__ void k_oz_offsets(Strided g, int d0, int d1, int64_t n, int64_t* __restrict__ off) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = x, o = 0;
    for (int d = d1 - 1; d >= d0; --d) {
      const int64_t e = g.ext[d];
      o += (r % e) * g.s1[d];
      r /= e;
    }
    off[x] = o;
  }
}

// one warp per row: e_r with max_k |X_rk| < 2^e_r (0 for a zero row, NONFINITE for Inf/NaN);
// element (row, k) at src[rowoff[row] + koff[k]].  Integer operations on the bit patterns
// (for finite values the order of |x| is the order of their sign-cleared patterns), so the
// pass does not queue on the FP64 pipe.
__global__ void k_oz_rowexp(const double* __restrict__ src, const int64_t* __restrict__ rowoff,
                            const int64_t* __restrict__ koff, int64_t K, int64_t rows, int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  for (int64_t row = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += (int64_t)gridDim.x * wpb) {
    const int64_t ro = rowoff[row];
    unsigned long long m = 0;
    for (int64_t k = lane; k < K; k += 32) m = max(m, (unsigned long long)__double_as_longlong(src[ro + koff[k]]) & kAbs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      int e = 0;
      if (m >= kInf) {
        e = NONFINITE;
      } else if (m != 0) {
        const int E = (int)(m >> 52);
        // |x| = 1.f 2^(E - 1023) = 0.1f 2^(E - 1022) < 2^(E - 1022); subnormals: below 2^-1022
        e = (E > 0) ? E - 1022 : -1022;
      }
      exps[row] = e;
    }
  }
}

// bf16 bit pattern of q * 2^(-7 s) for an integer |q| <= 64 (exact: at most 7 significant bits)
__device__ __forceinline__ unsigned short oz_slice_bits(long long q, int s) {
  if (q == 0) return 0;
  const unsigned int sign = q < 0 ? 0x8000u : 0u;
  const unsigned int a = (unsigned int)(q < 0 ? -q : q);
  const int p = 31 - __clz(a);  // a in [2^p, 2^(p+1))
  const unsigned int mant = (a << (7 - p)) & 0x7Fu;
  return (unsigned short)(sign | ((unsigned int)(127 + p - 7 * s) << 7) | mant);
}

// The 7 slices of x in a row with exponent e: y = x 2^(6 - e) (|y| < 64) held as the fixed-point
// integer Y = y 2^56 (|Y| < 2^62; bits of y below 2^-56 are dropped, far below the 2^-42 of
// the last slice), then q_s = round(Y / 2^56) (half up: |y - q_s| <= 1/2, so |q_s| <= 64 at
// every step) and Y = (Y - q_s 2^56) 128.  Integer operations only.  Subnormal inputs count as
// zero.
__device__ __forceinline__ void oz_slices(double x, int e, unsigned short (&out)[S]) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FFu);
  long long Y = 0;
  if (e != NONFINITE && E != 0) {
    const long long M = (long long)((u & ((1ull << 52) - 1)) | (1ull << 52));
    const int sh = E - 1013 - e;  // Y = M 2^sh; sh <= 9 because |x| < 2^e
    Y = sh >= 0 ? (M << sh) : (sh > -63 ? (M >> -sh) : 0);
    if (u >> 63) Y = -Y;
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const long long q = (Y + (1ll << 55)) >> 56;
    out[s] = oz_slice_bits(q, s);
    Y = (Y - (q << 56)) * 128;
  }
}

// the 7 slices of every element, padding rows and K zero: tiles of 32 rows x 64 k through
// shared memory, read along k (along_rows = 0) or along the rows (along_rows = 1) as the
// source is contiguous, written as bf16 pairs along k
__global__ void __launch_bounds__(256) k_oz_pack(const double* __restrict__ src, const int64_t* __restrict__ rowoff,
                                                 const int64_t* __restrict__ koff, int64_t rows, int64_t K,
                                                 int64_t rows_p, int64_t Kp, int along_rows,
                                                 const int* __restrict__ exps, __nv_bfloat16* __restrict__ dst) {
  __shared__ double tile[32][65];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t ktiles = Kp / 64, ntiles = (rows_p / 32) * ktiles;
  const int64_t plane = rows_p * Kp;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / ktiles) * 32, k0 = (t % ktiles) * 64;
    if (along_rows) {
      const int64_t r = r0 + tx;
      const int64_t ro = r < rows ? rowoff[r] : 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int kk = ty + 8 * i;
        const int64_t k = k0 + kk;
        tile[tx][kk] = (r < rows && k < K) ? src[ro + koff[k]] : 0.0;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = ty + 8 * i;
        const int64_t r = r0 + rr;
        const int64_t ro = r < rows ? rowoff[r] : 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kk = tx + 32 * h;
          const int64_t k = k0 + kk;
          tile[rr][kk] = (r < rows && k < K) ? src[ro + koff[k]] : 0.0;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = ty + 8 * i;
      const int64_t r = r0 + rr;
      const int e = r < rows ? exps[r] : NONFINITE;
      unsigned short q0[S], q1[S];
      oz_slices(tile[rr][2 * tx], e, q0);
      oz_slices(tile[rr][2 * tx + 1], e, q1);
      unsigned int* d = reinterpret_cast<unsigned int*>(dst + r * Kp + k0 + 2 * tx);
#pragma unroll
      for (int s = 0; s < S; ++s) d[s * (plane / 2)] = (unsigned int)q0[s] | ((unsigned int)q1[s] << 16);
    }
    __syncthreads();
  }
}

size_t operand_bytes(int64_t rows_p, int64_t Kp) { return (size_t)S * rows_p * Kp * 2 + (size_t)rows_p * 4 + 16; }

void pack(cudaStream_t st, const double* src, const Strided& g, int64_t rows, int64_t rows_p, int64_t K, int64_t Kp,
          void* buf) {
  if (rows < 1 || K < 1 || rows_p < rows || Kp < K || rows_p % 32 != 0 || Kp % 64 != 0)
    throw std::runtime_error("oz::pack: bad sizes");
  int* exps = exps_of(buf, rows_p, Kp);
  cudaMemsetAsync(exps, 0, (size_t)rows_p * 4, st);
  // the trailing dims whose extents multiply to K index K, the leading ones the rows
  int dk = g.ndim;
  for (int64_t prod = 1; dk > 0 && prod < K;) prod *= g.ext[--dk];
  int64_t* off = (int64_t*)dev_alloc((size_t)(rows + K) * sizeof(int64_t), st, true);
  int64_t k_inner = -1, r_inner = -1;
  for (int d = g.ndim - 1; d >= dk; --d)
    if (g.ext[d] > 1) {
      k_inner = g.s1[d];
      break;
    }
  for (int d = dk - 1; d >= 0; --d)
    if (g.ext[d] > 1) {
      r_inner = g.s1[d];
      break;
    }
  const int along_rows = (k_inner != 1 && r_inner == 1) ? 1 : 0;
  const int64_t ntiles = (rows_p / 32) * (Kp / 64);
  count_launches(4);
  k_oz_offsets<<<(int)std::min<int64_t>((rows + 255) / 256, 152 * 8), 256, 0, st>>>(g, 0, dk, rows, off);
  k_oz_offsets<<<(int)std::min<int64_t>((K + 255) / 256, 152 * 8), 256, 0, st>>>(g, dk, g.ndim, K, off + rows);
  k_oz_rowexp<<<(int)std::min<int64_t>((rows + 7) / 8, 152 * 16), 256, 0, st>>>(src, off, off + rows, K, rows, exps);
  k_oz_pack<<<(int)std::min<int64_t>(ntiles, 152 * 16), 256, 0, st>>>(src, off, off + rows, rows, K, rows_p, Kp,
                                                                      along_rows, exps, (__nv_bfloat16*)buf);
  dev_free(off, st, true);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("oz::pack launch: ") + cudaGetErrorString(e));
}

double gemm(cudaStream_t st, const void* a, int64_t Mp, const void* b, int64_t Np, int64_t Kp, int M, int N,
            double* C, int64_t sCm, int64_t sCn, double alpha, double beta, const Strided* om, const Strided* on,
            int nsplit_req, int* err, long long budget) {
  if (Mp % BM != 0 || Np % BN != 0 || Kp % BK != 0 || M < 1 || N < 1 || M > Mp || N > Np || Np / BN > 65535)
    throw std::runtime_error("oz::gemm: bad padding");
  if (beta != 0.0 && beta != 1.0) throw std::runtime_error("oz::gemm: beta must be 0 or 1");
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_dgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  CUtensorMap ta = tc::make_map(a, Mp, Kp, S, BM);
  CUtensorMap tb = tc::make_map(b, Np, Kp, S, BN);
  const int kt = (int)(Kp / BK);
  const int64_t tiles = (Mp / BM) * (Np / BN);
  const int chunks = (kt + KC_TILES - 1) / KC_TILES;
  int nsplit = nsplit_req;
  if (nsplit <= 0) {
    nsplit = 1;
    if (tiles < 152) nsplit = (int)std::min<int64_t>((152 + tiles - 1) / tiles, chunks);
    nsplit = std::min(nsplit, 64);
  }
  // at most 56 chunks (448 K tiles) per split keep the 64-bit accumulators below 2^62
  nsplit = std::max(nsplit, (kt + 447) / 448);
  nsplit = std::max(1, std::min(nsplit, kt));
  Params p;
  p.M = M;
  p.N = N;
  p.kt_total = kt;
  p.kt_per_split = (kt + nsplit - 1) / nsplit;
  nsplit = (kt + p.kt_per_split - 1) / p.kt_per_split;
  p.ea = exps_of(const_cast<void*>(a), Mp, Kp);
  p.eb = exps_of(const_cast<void*>(b), Np, Kp);
  p.C = C;
  p.sCm = sCm;
  p.sCn = sCn;
  p.part = nullptr;
  p.alpha = alpha;
  p.beta_zero = (beta == 0.0) ? 1 : 0;
  p.err = err;
  p.budget = budget;
  p.ostr = (om && on) ? 1 : 0;
  if (p.ostr) {
    p.om = *om;
    p.on = *on;
  } else {
    p.om.ndim = p.on.ndim = 0;
  }
  if (nsplit > 1) p.part = (double*)dev_alloc((size_t)nsplit * M * N * sizeof(double), st, true);
  if ((Mp / BM) * (Np / BN) > (int64_t)INT32_MAX) throw std::runtime_error("oz::gemm: too many tiles");
  p.mt = (int)(Mp / BM);
  p.nt = (int)(Np / BN);
  p.group_m = tc::raster_group(p.mt, BN);
  dim3 grid((unsigned)(p.mt * p.nt), 1u, (unsigned)nsplit);
  count_launches(1);
  k_tc_dgemm<<<grid, NTHREADS, SMEM_BYTES, st>>>(ta, tb, p);
  if (nsplit > 1) {
    launch_split_reduce_fp64(M, N, nsplit, p.part, C, sCm, sCn, p.beta_zero, p.ostr ? om : nullptr,
                             p.ostr ? on : nullptr, st);
    dev_free(p.part, st, true);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("oz::gemm launch: ") + cudaGetErrorString(e));
  return 2.0 * (double)Mp * (double)Np * (double)Kp * NPROD;
}

}  // namespace oz
}  // namespace ccsd
