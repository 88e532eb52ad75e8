// tcgen05 / TMA / mbarrier building blocks shared by the tensor-core kernels
// (inline PTX for sm_103a).  Every wait is bounded: mbar_wait gives up after its
// budget (TIMEOUT_CYCLES unless the launch passes a shorter one) or when another
// CTA has raised the error flag.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fpsplit.cuh"

namespace ccsd {
namespace tc {

constexpr int BM = 128, BK = 64;
constexpr long long TIMEOUT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity; false after `budget` clock cycles
// or when another CTA has raised the error flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* err,
                                          long long budget = TIMEOUT_CYCLES) {
  long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u) {
      if (*err) return false;
      if (clock64() - t0 > budget) return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // K-major operand tile, rows of 64 bf16 (128 B), 128-byte swizzle:
  // start address >> 4, leading-byte offset 16 B (unused with this swizzle),
  // stride-byte offset 1024 B between 8-row groups, descriptor version 1,
  // layout type 2 = SWIZZLE_128B.
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both K-major,
// N = BN (bits 17-22 hold N/8), M = 128 (bits 24-28 hold M/16).
template <int BN>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idsc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idsc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Grouped rasterisation of a 1-D grid over the mt x nt output tiles of a GEMM: consecutive
// CTAs take group_m row tiles of one column tile before moving on to the next column tile,
// so that the CTAs resident at the same time cover about group_m x (152 / group_m) tiles and
// share both operands' K strips through L2.  (Row tile fastest over the whole grid would
// give every resident CTA a private A strip: for the o^3 v^3 ring contractions that alone
// asks ~4 TB/s of DRAM at the tensor rate.)
__device__ __forceinline__ void raster_tile(int L, int mt, int nt, int group_m, int& tm, int& tn) {
  const int per_group = group_m * nt;
  const int g = L / per_group;
  const int first = g * group_m;
  const int gm = min(mt - first, group_m);
  const int r = L - g * per_group;
  tm = first + r % gm;
  tn = r / gm;
}

// Rows of tiles per raster group for a tile of 128 x bn: resident tiles about square in
// the bytes they read (group_m * 128 ~ (152 / group_m) * bn), at most mt.
inline int raster_group(int mt, int bn) {
  const int g = bn >= 256 ? 16 : (bn >= 128 ? 12 : 8);
  return mt < g ? mt : g;
}

// S bf16 slices of a pair of doubles (S = 2 or 3), x ~ slice 0 + slice 1 (+ slice 2), packed two
// per word (xa in the low half): slice 0 = bf16(hi), slice 1 = bf16((hi - slice 0) + lo),
// slice 2 = bf16 of that remainder, with (hi, lo) from double_to_float2.  Every FP32 remainder
// hi - slice is exact; the sum with lo rounds at 2^-32 |x|, so the three slices carry x to
// about 2^-26 |x| and two to 2^-17 |x|, the accuracy of the FP64 split x_0 = bf16(x),
// x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1).  Inf and NaN are carried by slice 0 alone.
__device__ __forceinline__ void split_bf16x2(double xa, double xb, int S, unsigned int (&out)[3]) {
  float ha, la, hb, lb;
  double_to_float2(xa, ha, la);
  double_to_float2(xb, hb, lb);
  __nv_bfloat162 b = __floats2bfloat162_rn(ha, hb);
  unsigned int w = *reinterpret_cast<unsigned int*>(&b);
  out[0] = w;
  // halves whose slice 0 is Inf or NaN (a non-finite x, or |x| beyond the bf16 range) keep
  // zero later slices
  const unsigned int finite = ((w & 0x7F80u) != 0x7F80u ? 0x0000FFFFu : 0u) |
                              ((w & 0x7F800000u) != 0x7F800000u ? 0xFFFF0000u : 0u);
  float ra = (ha - __uint_as_float(w << 16)) + la;
  float rb = (hb - __uint_as_float(w & 0xFFFF0000u)) + lb;
#pragma unroll
  for (int s = 1; s < 3; ++s) {
    if (s >= S) break;
    b = __floats2bfloat162_rn(ra, rb);
    w = *reinterpret_cast<unsigned int*>(&b) & finite;
    out[s] = w;
    ra -= __uint_as_float(w << 16);
    rb -= __uint_as_float(w & 0xFFFF0000u);
  }
}

// One double's S slices (the low halves of split_bf16x2).
__device__ __forceinline__ void split_bf16(double x, int S, unsigned short (&out)[3]) {
  unsigned int w[3] = {0u, 0u, 0u};
  split_bf16x2(x, 0.0, S, w);
  out[0] = (unsigned short)w[0];
  out[1] = (unsigned short)w[1];
  out[2] = (unsigned short)w[2];
}

// 3-D TMA map over bf16 slices [S][rows][Kp]: boxes of 64 K x box_rows rows x 1 slice,
// 128-byte swizzle (tc_gemm.cu)
CUtensorMap make_map(const void* base, int64_t rows, int64_t Kp, int S, int box_rows);

}  // namespace tc
}  // namespace ccsd
