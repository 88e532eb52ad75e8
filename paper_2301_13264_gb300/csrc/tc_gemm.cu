// Tensor-core (tcgen05) contraction path for the mixed-precision mode.
//
// An FP64 contraction C += alpha * A B^T (A: M x K, B: N x K) is evaluated as a
// sum of bf16 products: each FP64 operand is split into S bf16 slices
// x = x_0 + x_1 (+ x_2) (x_0 = bf16(x), x_1 = bf16(x - x_0), ...), and the
// products x_i y_j with i + j < S are accumulated in one FP32 TMEM accumulator
// (S = 2: 3 products, ~16 significant bits; S = 3: 6 products, ~24 bits before
// FP32 accumulation).  The slices live in a [S][rows][Kp] bf16 array (rows and
// K padded with zeros to the tile sizes) written by one gather kernel straight
// from the operand's strided FP64 layout; a 3-D TMA map selects the slice with
// its third coordinate, so the products are simply more K iterations of the
// same mainloop.
//
// Kernel (persistent, warp-specialised): at most one CTA per SM walks the work items
// (split-K part, 128 x BN output tile; BN = 64, 128 or 256) in raster groups, so that the
// CTAs resident at the same time share operand strips through L2.  Warp 0 lane 0 issues
// TMA loads into a 4- or 6-stage ring (mbarrier full/empty pairs); warp 1 lane 0 issues
// tcgen05.mma (kind::f16, bf16 inputs, FP32 accumulate, 128 x BN x 16 per instruction)
// into one of two TMEM accumulators and commits each stage back to the producer; warps
// 2..5 read a finished accumulator with tcgen05.ld, hand it back, and add alpha * acc
// into the FP64 output while the next item's products accumulate in the other one.
// When the output has few tiles the K iterations are split, and the partial tiles are
// summed in FP64 by a second kernel.  Every mbarrier wait is bounded; on timeout the
// kernel raises a device error flag, drains its own copies and MMAs (bounded), frees
// TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <utility>

#include "alloc.h"
#include "exec.h"
#include "fp64_tc.h"
#include "tcgen05.cuh"

namespace ccsd {

namespace tc {

constexpr int NTHREADS = 320;  // TMA warp, MMA warp, two groups of 4 epilogue warps
constexpr int A_BYTES = BM * BK * 2;
// per tile width BN (64, 128 or 256): B tile bytes, pipeline depth, shared memory
template <int BN>
struct Cfg {
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (BN == 256) ? 4 : 6;
  // stages, the strided-output column offsets [2][BN] (one row per epilogue group), barriers;
  // 1 KB alignment slack
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 2 * BN * 8 + 256 + 1024;
};
constexpr int MAXPROD = 6;

struct Params {
  int M, N;
  int kt_per_prod;    // 64-wide K tiles per slice
  int nprod;
  int it_per_split;   // K iterations per split
  int nsplit;         // K splits: work items are (split, tile) pairs
  int pa[MAXPROD], pb[MAXPROD];
  double* C;          // nsplit == 1: output
  long long sCm, sCn;
  double* part;       // nsplit > 1: partial tiles [split][M][N]
  double alpha;
  int beta_zero;
  int* err;
  // strided output (ostr != 0): element (m, n) lives at C + off(m; om) + off(n; on), where
  // off(x; g) decomposes x row-major over g.ext and sums the coordinates times g.s0
  int ostr;
  Strided om, on;
  int mt, nt, group_m;  // output tiles (rows, columns) and rows per raster group (raster_tile)
  long long budget;  // clock cycles a producer or MMA wait may take before the kernel gives up
  int stall;         // failure injection for tests: the producer issues no loads, so the MMA
                     // issuer's first wait runs out after `budget` and the kernel reports it
};

__device__ __forceinline__ long long dim_offset(long long x, const Strided& g) {
  long long off = 0;
  for (int d = g.ndim - 1; d >= 0; --d) {
    const long long e = g.ext[d];
    off += (x % e) * g.s0[d];
    x /= e;
  }
  return off;
}

// Named barrier among the 128 threads of epilogue group g (warps 2..5: barrier 1, warps 6..9:
// barrier 2); barrier 0 is __syncthreads.
__device__ __forceinline__ void epilogue_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent GEMM: gridDim.x CTAs (at most one per SM) walk the work items
// w = blockIdx.x, blockIdx.x + gridDim.x, ... of (split z, output tile) in raster order.
// Warp 0 lane 0 loads A and B K-tiles by TMA into the STAGES-deep ring; warp 1 lane 0
// issues the MMAs of an item into one of two TMEM accumulators (columns b*BN, b = item
// parity) and commits acc_full[b]; epilogue group b (warps 2..5 for b = 0, 6..9 for b = 1)
// reads the finished accumulator b (warp w owns TMEM lanes 32 (w % 4) ..), releases it with
// acc_empty[b] and writes the FP64 output.  The two groups write two tiles at once, doubling
// the loads and stores in flight for GEMMs whose output traffic decides their time, while
// the MMA warp fills whichever accumulator is free.
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, Params p) {
  constexpr int STAGES = Cfg<BN>::STAGES, B_BYTES = Cfg<BN>::B_BYTES, STAGE_BYTES = Cfg<BN>::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_skip;  // the error flag as thread 0 saw it: one decision for the whole CTA
  volatile int* err = p.err;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  long long* coloff = reinterpret_cast<long long*>(smem + STAGES * STAGE_BYTES);  // [2][BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES + 2 * BN * sizeof(long long));
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = p.mt * p.nt;
  const int items = tiles * p.nsplit;
  const int total = p.nprod * p.kt_per_prod;
  // K-iteration range of work item w (z = w / tiles)
  auto k_range = [&](int w, int& it0, int& it1) {
    const int z = w / tiles;
    it0 = z * p.it_per_split;
    it1 = min(total, it0 + p.it_per_split);
  };

  if (threadIdx.x == 0) {
    s_skip = *err;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf0, 1);
    mbar_init(accf0 + 8, 1);
    mbar_init(acce0, 4);
    mbar_init(acce0 + 8, 4);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tb)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (s_skip) {
    // an earlier kernel of this stream raised the flag: nothing to do but free TMEM
  } else if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      long long issued = 0;
      bool ok = true;
      for (int w = blockIdx.x; ok && w < items && !p.stall; w += gridDim.x) {
        int tm, tn, it0, it1;
        raster_tile(w % tiles, p.mt, p.nt, p.group_m, tm, tn);
        k_range(w, it0, it1);
        for (int it = it0; it < it1; ++it, ++issued) {
          const int s = (int)(issued % STAGES);
          const uint32_t ph = (uint32_t)(issued / STAGES) & 1u;
          if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err, p.budget)) {
            ok = false;
            break;
          }
          const int prod = it / p.kt_per_prod, kt = it % p.kt_per_prod;
          mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
          tma_load_3d(smem_u32(sA + s * A_BYTES), &ta, full0 + 8 * s, kt * BK, tm * BM, p.pa[prod]);
          tma_load_3d(smem_u32(sB + s * B_BYTES), &tb, full0 + 8 * s, kt * BK, tn * BN, p.pb[prod]);
        }
      }
      if (!ok) atomicExch((int*)p.err, 1);
      // the copies this CTA issued last (one per stage) must land before it exits
      for (long long it = issued - 1; it >= 0 && it >= issued - STAGES; --it) {
        const int s = (int)(it % STAGES);
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        const long long t0 = clock64();
        while (!mbar_try_wait(full0 + 8 * s, ph) && clock64() - t0 < TIMEOUT_CYCLES) {
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      long long consumed = 0;
      int item = 0;
      bool ok = true;
      for (int w = blockIdx.x; ok && w < items; w += gridDim.x, ++item) {
        int it0, it1;
        k_range(w, it0, it1);
        const int b = item & 1;
        const uint32_t use = (uint32_t)(item >> 1) & 1u;
        if (!mbar_wait(acce0 + 8 * b, use ^ 1u, err, p.budget)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        for (int it = it0; it < it1; ++it, ++consumed) {
          const int s = (int)(consumed % STAGES);
          const uint32_t ph = (uint32_t)(consumed / STAGES) & 1u;
          if (!mbar_wait(full0 + 8 * s, ph, err, p.budget)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
          for (int j = 0; j < BK / 16; ++j)
            mma_bf16(acc, smem_desc(a0 + 32 * j), smem_desc(b0 + 32 * j), idesc<BN>(), (it != it0 || j != 0) ? 1u : 0u);
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(accf0 + 8 * b);  // fires once the item's MMAs have completed
      }
      if (!ok) atomicExch((int*)p.err, 1);
      // every MMA this thread issued completes before the accumulators are freed
      mma_commit(done);
      const long long t0 = clock64();
      while (!mbar_try_wait(done, 0) && clock64() - t0 < TIMEOUT_CYCLES) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: group g = warps 2..5 (g = 0) or 6..9 (g = 1), the items of parity g,
    //      TMEM lanes 32 (warp % 4) of accumulator g ----
    const int g = (warp - 2) >> 2;
    const int lane_base = 32 * (warp & 3);
    const int et = threadIdx.x - 64 - 128 * g;  // 0..127
    long long* gcol = coloff + g * BN;
    int item = g;
    for (int w = blockIdx.x + g * gridDim.x; w < items; w += 2 * gridDim.x, item += 2) {
      int tm, tn, it0, it1;
      raster_tile(w % tiles, p.mt, p.nt, p.group_m, tm, tn);
      k_range(w, it0, it1);
      const int z = w / tiles;
      const int m0 = tm * BM, n0 = tn * BN;
      const int b = item & 1;
      const uint32_t use = (uint32_t)(item >> 1) & 1u;
      const bool split = p.nsplit > 1;
      const bool ostr = !split && p.ostr;
      // column offsets of a strided output for this tile (the previous tile's are no longer read)
      epilogue_sync(g);
      if (ostr)
        for (int c = et; c < BN; c += 128) gcol[c] = (n0 + c < p.N) ? dim_offset(n0 + c, p.on) : 0;
      epilogue_sync(g);
      // the accumulator wait spans the item's whole mainloop: default bound.  On failure the
      // group's four warps do not leave the loop (they would then disagree on the named
      // barrier above): they keep walking the items with every wait failing fast on the flag.
      const bool ready = mbar_wait(accf0 + 8 * b, use, err);
      if (!ready) atomicExch((int*)p.err, 1);
      fence_after();
      const int row = m0 + lane_base + lane;
      double* crow = split ? p.part + ((long long)z * p.M + row) * p.N
                           : (ostr ? p.C + (row < p.M ? dim_offset(row, p.om) : 0) : p.C + (long long)row * p.sCm);
      const long long cs = split ? 1 : p.sCn;
      const bool empty = it1 <= it0 || !ready;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        if (!empty) tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(b * BN + c), r);
        if (c + 32 >= BN) {
          // every load of this accumulator has completed: hand it back to the MMA warp
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive1(acce0 + 8 * b);
        }
        if (ready && row < p.M && !*err) {
          // read-modify-write of 32 distinct outputs: every load is issued before the first
          // store, so that they are in flight together (the compiler cannot know that the
          // strided destinations do not alias and would otherwise serialise them)
          const bool acc = !(split || p.beta_zero);
          double old[32];
          if (acc) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = n0 + c + j;
              old[j] = (n < p.N) ? crow[ostr ? gcol[c + j] : (long long)n * cs] : 0.0;
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int n = n0 + c + j;
            if (n < p.N) {
              const double v = empty ? 0.0 : p.alpha * (double)__uint_as_float(r[j]);
              crow[ostr ? gcol[c + j] : (long long)n * cs] = acc ? old[j] + v : v;
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
  }
}

// C[m, n] = sum_z part[z][m][n] (+ C[m, n] unless beta_zero); strided output as in Params
__global__ void k_tc_reduce(int M, int N, int nsplit, const double* __restrict__ part, double* C, long long sCm,
                            long long sCn, int beta_zero, int ostr, Strided om, Strided on) {
  const long long tot = (long long)M * N;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nsplit; ++z) s += part[(long long)z * tot + idx];
    const long long m = idx / N, n = idx % N;
    double* c = ostr ? C + dim_offset(m, om) + dim_offset(n, on) : C + m * sCm + n * sCn;
    *c = beta_zero ? s : (*c + s);
  }
}

// Offsets of a strided gather split into its leading (row) dims and its trailing (K)
// dims: off[x] = sum over dims d in [d0, d1) of coord_d(x) * g.s1[d], x decomposed
// row-major over those dims' extents.  One thread per entry.
__global__ void k_gather_offsets(Strided g, int d0, int d1, int64_t n, int64_t* __restrict__ off) {
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

// FP64 gather -> S bf16 slices dst[s][row][Kp] (rows_p x Kp, padding zero), element
// (row, k) read at src[rowoff[row] + koff[k]].  Tiles of 32 rows x 64 k through shared
// memory: along_rows = 0 reads consecutive k per warp (the source is contiguous along
// K), along_rows = 1 reads consecutive rows (contiguous along the rows) and transposes;
// the slices are written as bf16 pairs along k.
__global__ void __launch_bounds__(256) k_split_gather(const double* __restrict__ src, const int64_t* __restrict__ rowoff,
                                                      const int64_t* __restrict__ koff, int64_t rows, int64_t K,
                                                      int64_t rows_p, int64_t Kp, int S, int along_rows,
                                                      __nv_bfloat16* __restrict__ dst) {
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
    // split_bf16x2: integer and FP32 operations only (the FP64 pipe issues 2 per clock per SM)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = ty + 8 * i;
      unsigned int w[3];
      split_bf16x2(tile[rr][2 * tx], tile[rr][2 * tx + 1], S, w);
      unsigned int* d = reinterpret_cast<unsigned int*>(dst + (r0 + rr) * Kp + k0 + 2 * tx);
#pragma unroll
      for (int s = 0; s < 3; ++s)
        if (s < S) d[s * (plane / 2)] = w[s];
    }
    __syncthreads();
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      throw std::runtime_error("cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiled)p;
  }
  return fn;
}

CUtensorMap make_map(const void* base, int64_t rows, int64_t Kp, int S, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(rows * Kp * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

}  // namespace tc

struct Executor::CacheEntry {
  const double* src = nullptr;
  Strided g;
  int64_t rows_p = 0, K = 0;
  int S = 0;
  void* dev = nullptr;
  size_t bytes = 0;
};

static bool same_gather(const Strided& a, const Strided& b) {
  if (a.ndim != b.ndim) return false;
  for (int d = 0; d < a.ndim; ++d)
    if (a.ext[d] != b.ext[d] || a.s1[d] != b.s1[d]) return false;
  return true;
}

void Executor::drop_cache_range(const double* p, int64_t n) {
  bool dropped = false;
  for (size_t i = 0; i < cache_.size();) {
    CacheEntry* e = cache_[i];
    if (e->src >= p && e->src < p + n) {
      cudaStreamSynchronize(st_);  // no kernel may still read the slices
      dev_free(e->dev, st_, false);
      cache_bytes_ -= e->bytes;
      delete e;
      cache_.erase(cache_.begin() + i);
      dropped = true;
    } else {
      ++i;
    }
  }
  if (dropped) ++cache_epoch_;
}

void Executor::invalidate_frozen() {
  for (int t : frozen_tensors)
    if (ts_[t].p) drop_cache_range(ts_[t].p, numel(t));
}

void Executor::clear_cache() {
  for (CacheEntry* e : cache_) {
    dev_free(e->dev, st_, false);
    delete e;
  }
  cache_.clear();
  ++cache_epoch_;
  for (WPM& w : wpm_) {
    dev_free(w.plus, st_, false);
    dev_free(w.minus, st_, false);
  }
  wpm_.clear();
  if (pairs_) {
    dev_free(pairs_, st_, false);
    pairs_ = nullptr;
  }
  for (LadderTables& t : ladder_tables_) dev_free(t.dev, st_, false);
  ladder_tables_.clear();
  cache_bytes_ = 0;
  if (tc_err_) {
    dev_free(tc_err_, st_, false);
    tc_err_ = nullptr;
  }
}

int Executor::tc_error() {
  if (!tc_err_) return 0;
  int h = 0;
  if (cudaMemcpyAsync(&h, tc_err_, sizeof(int), cudaMemcpyDeviceToHost, st_) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(st_) != cudaSuccess) return -1;
  // a raised flag is reported once: lower it so that the next call's kernels run again
  if (h != 0 && cudaMemsetAsync(tc_err_, 0, sizeof(int), st_) != cudaSuccess) return -1;
  return h;
}

// bf16 slices [S][rows_p][Kp] of an FP64 operand given as a strided gather over
// (row dims..., K dims...); padding rows and columns are zero.  rows_p is a multiple of
// 128 and Kp of 64, so the 32 x 64 tiles of the gather cover the array exactly.
static __nv_bfloat16* make_slices(cudaStream_t st, const double* src, const Strided& g, int64_t rows, int64_t rows_p,
                                  int64_t K, int S, int64_t Kp) {
  size_t bytes = (size_t)S * rows_p * Kp * sizeof(__nv_bfloat16);
  void* p = dev_alloc(bytes, st, true);
  // the trailing dims whose extents multiply to K index K, the leading ones the rows
  int dk = g.ndim;
  for (int64_t prod = 1; dk > 0 && prod < K;) prod *= g.ext[--dk];
  int64_t* off = (int64_t*)dev_alloc((size_t)(rows + K) * sizeof(int64_t), st, true);
  count_launches(3);
  tc::k_gather_offsets<<<(int)std::min<int64_t>((rows + 255) / 256, 152 * 8), 256, 0, st>>>(g, 0, dk, rows, off);
  tc::k_gather_offsets<<<(int)std::min<int64_t>((K + 255) / 256, 152 * 8), 256, 0, st>>>(g, dk, g.ndim, K, off + rows);
  // read along whichever side is contiguous in the source
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
  tc::k_split_gather<<<(int)std::min<int64_t>(ntiles, 152 * 16), 256, 0, st>>>(
      src, off, off + rows, rows, K, rows_p, Kp, S, along_rows, (__nv_bfloat16*)p);
  dev_free(off, st, true);
  return (__nv_bfloat16*)p;
}

// multiprocessors of the current device (queried once per device)
static int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

template <int BN>
static void launch_tc(dim3 grid, const CUtensorMap& ta, const CUtensorMap& tb, const tc::Params& p, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Cfg<BN>::SMEM_BYTES);
    attr = true;
  }
  count_launches(1);
  tc::k_tc_gemm<BN><<<grid, tc::NTHREADS, tc::Cfg<BN>::SMEM_BYTES, st>>>(ta, tb, p);
}

// Output stride between consecutive indices of one side of a GEMM: the stride of that side's
// fastest-varying dimension (offset table g), or the direct stride.
static int64_t lane_stride(const Strided* g, int64_t direct) {
  if (!g) return direct < 0 ? -direct : direct;
  for (int d = g->ndim - 1; d >= 0; --d)
    if (g->ext[d] > 1) return g->s0[d] < 0 ? -g->s0[d] : g->s0[d];
  return 0;
}

bool Executor::tc_contract(int M, int N, int K, const double* A, const Strided& Ag, const double* B,
                           const Strided& Bg, double* C, int64_t sCm, int64_t sCn, double alpha, double beta,
                           bool a_const, bool b_const, const Strided* om, const Strided* on) {
  if (prec_ == PREC_FP64_TC) return fp64tc_contract(M, N, K, A, Ag, B, Bg, C, sCm, sCn, alpha, beta, a_const, b_const, om, on);
  if (M < 1 || N < 1 || K < 1) return false;
  if (beta != 0.0 && beta != 1.0) return false;
  Strided ag = Ag, bg = Bg;
  // the MMA tile is 128 rows of A by BN rows of B: put the longer side on A
  if (M < tc::BM && N > M) {
    std::swap(M, N);
    std::swap(A, B);
    std::swap(ag, bg);
    std::swap(a_const, b_const);
    std::swap(sCm, sCn);
    std::swap(om, on);
  }
  // the epilogue's 32 lanes hold 32 consecutive rows m: give the M side the output dimension
  // with the smaller stride, so that their stores coalesce
  if (N >= tc::BM && lane_stride(om, sCm) > lane_stride(on, sCn)) {
    std::swap(M, N);
    std::swap(A, B);
    std::swap(ag, bg);
    std::swap(a_const, b_const);
    std::swap(sCm, sCn);
    std::swap(om, on);
  }
  const int S = (splits_ >= 3) ? 3 : 2;
  const int64_t Kp = ((int64_t)K + tc::BK - 1) / tc::BK * tc::BK;
  const int64_t Mp = ((int64_t)M + tc::BM - 1) / tc::BM * tc::BM;
  const TcChoice ch = tc_choice(M, N, Kp, S, om && on);
  const int BN = ch.bn;
  const int64_t Np = ((int64_t)N + BN - 1) / BN * BN;
  if (Np / BN > 65535) return false;
  if (!tc_err_) {
    tc_err_ = (int*)dev_alloc(sizeof(int), st_, false);
    cudaMemsetAsync(tc_err_, 0, sizeof(int), st_);
  }
  auto get = [&](const double* src, const Strided& g, int64_t rows, int64_t rows_p, bool cst, bool& owned) {
    if (cst) {
      for (CacheEntry* e : cache_)
        if (e->src == src && same_gather(e->g, g) && e->rows_p == rows_p && e->K == K && e->S == S) {
          owned = false;
          return (__nv_bfloat16*)e->dev;
        }
    }
    __nv_bfloat16* p = make_slices(st_, src, g, rows, rows_p, K, S, Kp);
    owned = !cst;
    if (cst) {
      dev_keep(p);  // a cache entry: lives until the cache drops it
      CacheEntry* e = new CacheEntry{src, g, rows_p, (int64_t)K, S, p, (size_t)S * rows_p * Kp * 2};
      cache_.push_back(e);
      cache_bytes_ += e->bytes;
    }
    return p;
  };
  bool ownA = false, ownB = false;
  __nv_bfloat16* a = get(A, ag, M, Mp, a_const, ownA);
  __nv_bfloat16* b = get(B, bg, N, Np, b_const, ownB);
  tc_run(a, Mp, b, Np, K, Kp, S, M, N, C, sCm, sCn, alpha, beta, om, on, BN, ch.nsplit);
  if (ownA) dev_free(a, st_, true);
  if (ownB) dev_free(b, st_, true);
  return true;
}

bool Executor::fp64tc_contract(int M, int N, int K, const double* A, const Strided& Ag, const double* B,
                               const Strided& Bg, double* C, int64_t sCm, int64_t sCn, double alpha, double beta,
                               bool a_const, bool b_const, const Strided* om, const Strided* on) {
  if (M < 1 || N < 1 || K < 1) return false;
  if (beta != 0.0 && beta != 1.0) return false;
  Strided ag = Ag, bg = Bg;
  if (M < tc::BM && N > M) {
    std::swap(M, N);
    std::swap(A, B);
    std::swap(ag, bg);
    std::swap(a_const, b_const);
    std::swap(sCm, sCn);
    std::swap(om, on);
  }
  const int64_t Kp = ((int64_t)K + tc::BK - 1) / tc::BK * tc::BK;
  const int64_t Mp = ((int64_t)M + tc::BM - 1) / tc::BM * tc::BM;
  const int64_t Np = ((int64_t)N + oz::BN - 1) / oz::BN * oz::BN;
  if (Np / oz::BN > 65535) return false;
  if (!tc_err_) {
    tc_err_ = (int*)dev_alloc(sizeof(int), st_, false);
    cudaMemsetAsync(tc_err_, 0, sizeof(int), st_);
  }
  auto get = [&](const double* src, const Strided& g, int64_t rows, int64_t rows_p, bool cst, bool& owned) {
    if (cst) {
      for (CacheEntry* e : cache_)
        if (e->src == src && same_gather(e->g, g) && e->rows_p == rows_p && e->K == K && e->S == oz::S) {
          owned = false;
          return e->dev;
        }
    }
    const size_t bytes = oz::operand_bytes(rows_p, Kp);
    void* p = dev_alloc(bytes, st_, true);
    oz::pack(st_, src, g, rows, rows_p, K, Kp, p);
    owned = !cst;
    if (cst) {
      dev_keep(p);  // a cache entry: lives until the cache drops it
      CacheEntry* e = new CacheEntry{src, g, rows_p, (int64_t)K, oz::S, p, bytes};
      cache_.push_back(e);
      cache_bytes_ += e->bytes;
    }
    return p;
  };
  bool ownA = false, ownB = false;
  void* a = get(A, ag, M, Mp, a_const, ownA);
  void* b = get(B, bg, N, Np, b_const, ownB);
  last_tc_issued = oz::gemm(st_, a, Mp, b, Np, Kp, M, N, C, sCm, sCn, alpha, beta, om, on, 0, tc_err_,
                            wait_cycles > 0 ? wait_cycles : tc::TIMEOUT_CYCLES);
  if (ownA) dev_free(a, st_, true);
  if (ownB) dev_free(b, st_, true);
  return true;
}

static int tile_width(int N) { return (N > 128) ? 256 : (N > 64 ? 128 : 64); }

// split-K count that fills the machine when the output has few tiles
static int split_count(int64_t tiles, int iters) {
  int nsplit = 1;
  if (tiles < 148 && iters >= 32) nsplit = (int)std::min<int64_t>(std::min<int64_t>(296 / tiles, iters / 16), 64);
  return std::max(nsplit, 1);
}

Executor::TcChoice Executor::tc_choice(int M, int N, int64_t Kp, int S, bool strided) {
  TcChoice ch{tile_width(N), 0};
  if (!autotune) return ch;
  const std::array<int64_t, 4> key{M, N, Kp, S * 2 + (strided ? 1 : 0)};
  auto it = tc_tuned_.find(key);
  if (it != tc_tuned_.end()) return it->second;
  if (capturing) return ch;  // shapes are tuned in an uncaptured run first
  // candidates: tile widths up to twice the output width, split counts around the heuristic
  const int64_t Mp = ((int64_t)M + tc::BM - 1) / tc::BM * tc::BM;
  const int64_t Nmax = ((int64_t)N + 255) / 256 * 256;
  void *a = nullptr, *b = nullptr;
  double* C = nullptr;
  const size_t abytes = (size_t)S * Mp * Kp * 2, bbytes = (size_t)S * Nmax * Kp * 2;
  try {
    a = dev_alloc(abytes, st_, false);
    b = dev_alloc(bbytes, st_, false);
    C = (double*)dev_alloc((size_t)M * N * sizeof(double), st_, false);
  } catch (const OutOfMemory&) {
    dev_free(a, st_, false);
    dev_free(b, st_, false);
    return ch;  // no room to tune: keep the heuristic
  }
  cudaMemsetAsync(a, 0, abytes, st_);
  cudaMemsetAsync(b, 0, bbytes, st_);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int nprod = (S == 2) ? 3 : 6;
  const int iters = nprod * (int)(Kp / tc::BK);
  float best = 1e30f;
  for (int bn : {64, 128, 256}) {
    if (bn > 64 && bn >= 2 * N) continue;
    const int64_t Np = ((int64_t)N + bn - 1) / bn * bn;
    const int64_t tiles = (Mp / tc::BM) * (Np / bn);
    const int h = split_count(tiles, iters);
    std::vector<int> splits{1, h, std::min(2 * h, std::max(1, iters / 4))};
    if (tiles < 152 && iters >= 8) splits.push_back(std::max(1, std::min<int>(152 / (int)tiles, iters / 4)));
    std::sort(splits.begin(), splits.end());
    splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
    for (int ns : splits) {
      if (ns > 64) continue;
      tc_run(a, Mp, b, Np, (int)Kp, Kp, S, M, N, C, N, 1, 1.0, 0.0, nullptr, nullptr, bn, ns);  // warm
      cudaEventRecord(e0, st_);
      for (int r = 0; r < 3; ++r)
        tc_run(a, Mp, b, Np, (int)Kp, Kp, S, M, N, C, N, 1, 1.0, 0.0, nullptr, nullptr, bn, ns);
      cudaEventRecord(e1, st_);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        ch = TcChoice{bn, ns};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st_);
  dev_free(a, st_, false);
  dev_free(b, st_, false);
  dev_free(C, st_, false);
  tc_tuned_[key] = ch;
  return ch;
}

void Executor::tc_run(const void* a, int64_t Mp, const void* b, int64_t Np, int K, int64_t Kp, int S, int M, int N,
                      double* C, int64_t sCm, int64_t sCn, double alpha, double beta, const Strided* om,
                      const Strided* on, int BN, int nsplit_req) {
  (void)K;
  if (BN == 0) BN = tile_width(N);
  if (Np % BN != 0 || Mp % tc::BM != 0 || Np / BN > 65535) throw std::runtime_error("tc_run: bad padding");
  if (!tc_err_) {
    tc_err_ = (int*)dev_alloc(sizeof(int), st_, false);
    cudaMemsetAsync(tc_err_, 0, sizeof(int), st_);
  }
  CUtensorMap ta = tc::make_map(a, Mp, Kp, S, tc::BM);
  CUtensorMap tb = tc::make_map(b, Np, Kp, S, BN);
  tc::Params p;
  p.M = M;
  p.N = N;
  p.kt_per_prod = (int)(Kp / tc::BK);
  // products x_i y_j with i + j < S
  const int pa3[3] = {0, 0, 1}, pb3[3] = {0, 1, 0};
  const int pa6[6] = {0, 0, 1, 0, 1, 2}, pb6[6] = {0, 1, 0, 2, 1, 0};
  p.nprod = (S == 2) ? 3 : 6;
  for (int i = 0; i < p.nprod; ++i) {
    p.pa[i] = (S == 2) ? pa3[i] : pa6[i];
    p.pb[i] = (S == 2) ? pb3[i] : pb6[i];
  }
  const int iters = p.nprod * p.kt_per_prod;
  const int64_t tiles = (Mp / tc::BM) * (Np / BN);
  int nsplit = nsplit_req > 0 ? std::min(nsplit_req, iters) : split_count(tiles, iters);
  p.it_per_split = (iters + nsplit - 1) / nsplit;
  nsplit = (iters + p.it_per_split - 1) / p.it_per_split;
  p.C = C;
  p.sCm = sCm;
  p.sCn = sCn;
  p.part = nullptr;
  p.alpha = alpha;
  p.beta_zero = (beta == 0.0) ? 1 : 0;
  p.err = tc_err_;
  p.ostr = (om && on) ? 1 : 0;
  if (p.ostr) {
    p.om = *om;
    p.on = *on;
  } else {
    p.om.ndim = p.on.ndim = 0;
  }
  p.budget = wait_cycles > 0 ? wait_cycles : tc::TIMEOUT_CYCLES;
  p.stall = stall_next ? 1 : 0;
  stall_next = false;
  if (nsplit > 1) p.part = (double*)dev_alloc((size_t)nsplit * M * N * sizeof(double), st_, true);
  if ((Mp / tc::BM) * (Np / BN) > (int64_t)INT32_MAX) throw std::runtime_error("tc_run: too many tiles");
  p.mt = (int)(Mp / tc::BM);
  p.nt = (int)(Np / BN);
  p.group_m = tc::raster_group(p.mt, BN);
  p.nsplit = nsplit;
  if ((int64_t)p.mt * p.nt * nsplit > (int64_t)INT32_MAX) throw std::runtime_error("tc_run: too many work items");
  // persistent: at most one CTA per SM walks the (split, tile) work items
  const int items = p.mt * p.nt * nsplit;
  dim3 grid((unsigned)std::min(items, sm_count()), 1u, 1u);
  last_tc_issued = 2.0 * (double)Mp * (double)Np * (double)Kp * p.nprod;
  if (BN == 256)
    launch_tc<256>(grid, ta, tb, p, st_);
  else if (BN == 128)
    launch_tc<128>(grid, ta, tb, p, st_);
  else
    launch_tc<64>(grid, ta, tb, p, st_);
  if (nsplit > 1) {
    const long long tot = (long long)M * N;
    count_launches(1);
    tc::k_tc_reduce<<<(int)std::min<long long>((tot + 255) / 256, 152 * 16), 256, 0, st_>>>(
        M, N, nsplit, p.part, C, sCm, sCn, p.beta_zero, p.ostr, p.om, p.on);
    dev_free(p.part, st_, true);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("tc gemm launch: ") + cudaGetErrorString(e));
}

void launch_split_reduce_fp64(int M, int N, int nsplit, const double* part, double* C, long long sCm, long long sCn,
                              int beta_zero, const Strided* om, const Strided* on, cudaStream_t st) {
  const long long tot = (long long)M * N;
  Strided gm, gn;
  gm.ndim = gn.ndim = 0;
  if (om && on) {
    gm = *om;
    gn = *on;
  }
  count_launches(1);
  tc::k_tc_reduce<<<(int)std::min<long long>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(
      M, N, nsplit, part, C, sCm, sCn, beta_zero, (om && on) ? 1 : 0, gm, gn);
}

}  // namespace ccsd
