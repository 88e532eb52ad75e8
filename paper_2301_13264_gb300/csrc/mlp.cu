// Learned initial guess for the doubles amplitudes: a 3 -> 128 -> 128 -> 1 MLP
// (tanh hidden layers) mapping per-element MP2-type features
//   x = (t_MP2_ijab, D_ijab, |(ia|jb)|),  t_MP2 = -(ia|jb) / D,  D = e_a + e_b - e_i - e_j,
// to the correction t_CCSD - t_MP2.  Training (MSE loss, Adam) and inference run
// in these kernels: one CTA of 128 threads handles tiles of 8 rows, thread k owns
// hidden unit k; W2 sits in shared memory with padded rows (conflict-free row and
// column access), per-CTA gradient sums are added to global memory at the end.
// Arithmetic is FP32; inference uses the weights rounded to bf16 (FP32 accumulate).
//
// Model array layout (floats), MLP_PARAMS in total:
//   W1[128][3], b1[128], W2[128][128], b2[128], w3[128], b3,
//   feature mean[3], feature scale[3], target scale.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <vector>

#include "exec.h"
#include "kernels.cuh"
#include "mlp.h"
#include "tcgen05.cuh"

namespace ccsd {
namespace mlp {

constexpr int H = 128, TR = 8, P2 = H + 1;
constexpr int OW1 = 0, OB1 = OW1 + H * 3, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
constexpr int NW = OB3 + 1;  // trainable parameters
constexpr int OMEAN = NW, OSCALE = NW + 3, OTSCALE = NW + 6;
static_assert(OTSCALE + 1 == kParams, "layout");
static_assert(NW == kTrainable, "layout");

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16(x)); }

// mode 0: inference (out[r] = prediction in target units); mode 1: loss + gradients.
// X[r][3] raw features, T[r] raw targets (mode 1), grad[NW] accumulated (mode 1), loss[0] += sum sq.
template <int MODE>
__global__ void __launch_bounds__(H) k_mlp(const float* __restrict__ model, const float* __restrict__ X,
                                           const float* __restrict__ T, const int64_t* __restrict__ idx, int64_t n,
                                           float inv_n, float* __restrict__ out, float* __restrict__ grad,
                                           float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* W2 = sm;                  // [H][P2]
  float* dW2 = W2 + H * P2;        // [H][P2] (mode 1)
  float* h1 = dW2 + (MODE ? H * P2 : 0);
  float* h2 = h1 + TR * H;
  float* dz = h2 + TR * H;
  float* xs = dz + TR * H;         // [TR][3]
  float* ys = xs + TR * 4;         // [TR]
  float* red = ys + TR;            // [TR][4]
  const int k = threadIdx.x, warp = k >> 5, lane = k & 31;
  const bool q = (MODE == 0);      // inference uses bf16-rounded weights
  for (int e = k; e < H * H; e += H) {
    const float w = model[OW2 + e];
    W2[(e / H) * P2 + (e % H)] = q ? round_bf16(w) : w;
    if (MODE) dW2[(e / H) * P2 + (e % H)] = 0.f;
  }
  float w1[3];
  for (int d = 0; d < 3; ++d) w1[d] = q ? round_bf16(model[OW1 + k * 3 + d]) : model[OW1 + k * 3 + d];
  const float b1 = q ? round_bf16(model[OB1 + k]) : model[OB1 + k];
  const float b2 = q ? round_bf16(model[OB2 + k]) : model[OB2 + k];
  const float w3 = q ? round_bf16(model[OW3 + k]) : model[OW3 + k];
  const float b3 = q ? round_bf16(model[OB3]) : model[OB3];
  float mean[3], scale[3];
  for (int d = 0; d < 3; ++d) {
    mean[d] = model[OMEAN + d];
    scale[d] = model[OSCALE + d];
  }
  const float tscale = model[OTSCALE];
  float gw1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  __syncthreads();
  const int64_t ntiles = (n + TR - 1) / TR;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TR;
    if (k < TR * 3) {
      const int r = k / 3, d = k % 3;
      const int64_t row = r0 + r;
      float v = 0.f;
      if (row < n) {
        const int64_t src = idx ? idx[row] : row;
        v = (X[src * 3 + d] - mean[d]) / scale[d];
      }
      xs[r * 4 + d] = v;
    }
    __syncthreads();
    for (int r = 0; r < TR; ++r) {
      const float z = w1[0] * xs[r * 4] + w1[1] * xs[r * 4 + 1] + w1[2] * xs[r * 4 + 2] + b1;
      h1[r * H + k] = tanhf(z);
    }
    __syncthreads();
    for (int r = 0; r < TR; ++r) {
      float z = b2;
      const float* hr = h1 + r * H;
      const float* wr = W2 + k * P2;
#pragma unroll 8
      for (int j = 0; j < H; ++j) z = fmaf(wr[j], hr[j], z);
      const float a = tanhf(z);
      h2[r * H + k] = a;
      float part = w3 * a;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
      if (lane == 0) red[r * 4 + warp] = part;
    }
    __syncthreads();
    if (k < TR) {
      ys[k] = red[k * 4] + red[k * 4 + 1] + red[k * 4 + 2] + red[k * 4 + 3] + b3;
      const int64_t row = r0 + k;
      if (MODE == 0 && row < n) out[idx ? idx[row] : row] = ys[k] * tscale;
    }
    __syncthreads();
    if (MODE == 1) {
      // dL/dy for L = inv_n * sum (y - t/tscale)^2 in normalised target units
      for (int r = 0; r < TR; ++r) {
        const int64_t row = r0 + r;
        float dy = 0.f;
        if (row < n) {
          const int64_t src = idx ? idx[row] : row;
          const float diff = ys[r] - T[src] / tscale;
          dy = 2.f * inv_n * diff;
          if (k == 0) lsum += diff * diff;
        }
        const float a = h2[r * H + k];
        gw3 += dy * a;
        if (k == 0) gb3 += dy;
        const float g = dy * w3 * (1.f - a * a);
        dz[r * H + k] = g;
        gb2 += g;
      }
      __syncthreads();
      // dW2[k][j] += sum_r dz[r][k] h1[r][j]
      for (int r = 0; r < TR; ++r) {
        const float g = dz[r * H + k];
        if (g != 0.f) {
          float* dr = dW2 + k * P2;
          const float* hr = h1 + r * H;
          for (int j = 0; j < H; ++j) dr[j] = fmaf(g, hr[j], dr[j]);
        }
      }
      // thread k as input unit j = k: dh1[r][j] = sum_i W2[i][j] dz[r][i]
      for (int r = 0; r < TR; ++r) {
        float s = 0.f;
        for (int i = 0; i < H; ++i) s = fmaf(W2[i * P2 + k], dz[r * H + i], s);
        const float a = h1[r * H + k];
        const float g1 = s * (1.f - a * a);
        gb1 += g1;
        for (int d = 0; d < 3; ++d) gw1[d] += g1 * xs[r * 4 + d];
      }
    }
    __syncthreads();
  }
  if (MODE == 1) {
    for (int d = 0; d < 3; ++d) atomicAdd(&grad[OW1 + k * 3 + d], gw1[d]);
    atomicAdd(&grad[OB1 + k], gb1);
    atomicAdd(&grad[OB2 + k], gb2);
    atomicAdd(&grad[OW3 + k], gw3);
    if (k == 0) {
      atomicAdd(&grad[OB3], gb3);
      atomicAdd(loss, lsum * inv_n);
    }
    __syncthreads();
    for (int e = k; e < H * H; e += H) atomicAdd(&grad[OW2 + e], dW2[(e / H) * P2 + (e % H)]);
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// uniform minibatch indices from a counter-based hash (splitmix64 of seed, step, slot)
__global__ void k_sample(int64_t* idx, int batch, int64_t n, unsigned long long seed, unsigned long long step) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (step * 1315423911ull + (unsigned long long)i + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  idx[i] = (int64_t)(z % (unsigned long long)n);
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores.  One CTA of 128 threads owns a 128-row tile at a
// time (persistent over tiles): thread t computes row t's first layer in FP32,
// rounds h1 to bf16 and writes it into the A operand in the 128-byte-swizzled
// K-major layout a TMA copy would produce (two 64-wide K chunks); W2 sits in the
// same layout as the B operand for the CTA's life.  One elected thread issues the
// 128 x 128 x 128 product as 8 tcgen05.mma (kind::f16, FP32 accumulate in TMEM);
// after the commit barrier each warp reads its 32 TMEM lanes (= rows) and applies
// tanh, w3 and b3 in registers.  Waits are bounded; on timeout the kernel raises
// the error flag and leaves.
// ---------------------------------------------------------------------------
constexpr int TILE_BYTES = 128 * 64 * 2;  // one 128-row x 64-column bf16 chunk

// tanh(x) = 1 - 2 / (exp(2x) + 1) with the hardware base-2 exponential and reciprocal
// approximations (absolute error ~1e-7, below the bf16 spacing of the activations);
// |x| is clamped at 9, where tanh is 1 to FP32 precision.
__device__ __forceinline__ float fast_tanh(float x) {
  const float xc = fminf(fmaxf(x, -9.f), 9.f);
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(xc * 2.8853900817779268f));  // 2 / ln 2
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.f));
  return fmaf(-2.f, r, 1.f);
}

// byte offset of element (row, k) (k < 64) in a 128B-swizzled chunk
__device__ __forceinline__ uint32_t swz(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ row) & 7) << 4) + ((k & 7) << 1));
}

__global__ void __launch_bounds__(H, 2)
    k_mlp_infer_tc(const float* __restrict__ model, const float* __restrict__ X, int64_t n, float* __restrict__ out,
                   int* err) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;                  // 2 chunks: h1 [128 rows][128 k]
  uint8_t* sB = sm + 2 * TILE_BYTES;  // 2 chunks: W2 [128 out][128 in]
  float* par = (float*)(sm + 4 * TILE_BYTES);  // W1[128][3], b1, b2, w3 (bf16-rounded)
  float* sW1 = par;
  float* sb1 = par + 3 * H;
  float* sb2 = sb1 + H;
  float* sw3 = sb2 + H;
  uint64_t* bar = (uint64_t*)(sw3 + H);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  if (*(volatile int*)err) return;
  for (int e = t; e < H * H; e += H) {
    const int j = e / H, k = e % H;
    *(__nv_bfloat16*)(sB + (k >> 6) * TILE_BYTES + swz(j, k & 63)) = __float2bfloat16(model[OW2 + e]);
  }
  for (int e = t; e < 3 * H; e += H) sW1[e] = round_bf16(model[OW1 + e]);
  sb1[t] = round_bf16(model[OB1 + t]);
  sb2[t] = round_bf16(model[OB2 + t]);
  sw3[t] = round_bf16(model[OW3 + t]);
  const float b3 = round_bf16(model[OB3]);
  float mean[3], scale[3];
  for (int d = 0; d < 3; ++d) {
    mean[d] = model[OMEAN + d];
    scale[d] = model[OSCALE + d];
  }
  const float tscale = model[OTSCALE];
  const uint32_t mbar = tc::smem_u32(bar);
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                 "r"(H)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const int64_t ntiles = (n + H - 1) / H;
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t row = tile * H + t;
    float x[3] = {0.f, 0.f, 0.f};
    if (row < n)
      for (int d = 0; d < 3; ++d) x[d] = (X[row * 3 + d] - mean[d]) / scale[d];
    // first layer -> bf16 A operand, 8 units (one 16-byte chunk) at a time
    for (int k0 = 0; k0 < H; k0 += 8) {
      uint32_t pk[4];
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 2 * q;
        const float h0 = fast_tanh(sW1[k * 3] * x[0] + sW1[k * 3 + 1] * x[1] + sW1[k * 3 + 2] * x[2] + sb1[k]);
        const float h1 = fast_tanh(sW1[(k + 1) * 3] * x[0] + sW1[(k + 1) * 3 + 1] * x[1] + sW1[(k + 1) * 3 + 2] * x[2] +
                                   sb1[k + 1]);
        __nv_bfloat162 v = __floats2bfloat162_rn(h0, h1);
        pk[q] = *reinterpret_cast<uint32_t*>(&v);
      }
      *reinterpret_cast<uint4*>(sA + (k0 >> 6) * TILE_BYTES + swz(t, k0 & 63)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (t == 0) {
      tc::fence_after();
      for (int kc = 0; kc < 2; ++kc)
        for (int j = 0; j < 4; ++j)
          tc::mma_bf16(tmem, tc::smem_desc(tc::smem_u32(sA + kc * TILE_BYTES) + 32 * j),
                       tc::smem_desc(tc::smem_u32(sB + kc * TILE_BYTES) + 32 * j), tc::idesc<H>(),
                       (kc | j) != 0 ? 1u : 0u);
      tc::mma_commit(mbar);
    }
    __syncwarp();
    ok = tc::mbar_wait(mbar, phase, err);
    phase ^= 1u;
    tc::fence_after();
    if (!ok) {
      atomicExch(err, 1);
      // the product may still be running: give it a bounded second wait before TMEM is freed
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(mbar, phase ^ 1u) && clock64() - t0 < tc::TIMEOUT_CYCLES) {
      }
      break;
    }
    float y = b3;
    for (int c = 0; c < H; c += 32) {
      uint32_t r[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
#pragma unroll
      for (int j = 0; j < 32; ++j) y = fmaf(sw3[c + j], fast_tanh(__uint_as_float(r[j]) + sb2[c + j]), y);
    }
    if (row < n) out[row] = y * tscale;
    tc::fence_before();
    __syncthreads();  // A tile and accumulator are reused by the next tile
    tc::fence_after();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H) : "memory");
}

constexpr size_t kInferSmem = 1024 + 4 * TILE_BYTES + 6 * H * sizeof(float) + 64;

size_t smem_bytes(int mode) { return sizeof(float) * ((mode ? 2 : 1) * H * P2 + 3 * TR * H + TR * 4 + TR + TR * 4); }

static int grid_for_rows(int64_t n) {
  int64_t t = (n + TR - 1) / TR;
  return (int)std::max<int64_t>(1, std::min<int64_t>(t, 152 * 4));
}

__device__ int g_mlp_err = 0;

void predict(const float* model, const float* X, int64_t n, float* out, cudaStream_t st) {
  static bool attr = false;
  static int* err = nullptr;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
    cudaGetSymbolAddress((void**)&err, g_mlp_err);
    attr = true;
  }
  const int64_t tiles = (n + H - 1) / H;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 2));
  count_launches(1);
  k_mlp_infer_tc<<<grid, H, kInferSmem, st>>>(model, X, n, out, err);
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    throw DeviceTimeout("a tensor-core wait in the MLP inference kernel exceeded its budget");
  }
}

void gradient(const float* model, const float* X, const float* T, const int64_t* idx, int64_t n, float* grad,
              float* loss, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(1));
    attr = true;
  }
  cudaMemsetAsync(grad, 0, NW * sizeof(float), st);
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  count_launches(1);
  const int grid = std::min(grid_for_rows(n), 128);  // fewer CTAs: fewer gradient atomics
  k_mlp<1><<<grid, H, smem_bytes(1), st>>>(model, X, T, idx, n, 1.f / (float)n, nullptr, grad, loss);
}

void adam(float* w, const float* g, float* m, float* v, float lr, int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  count_launches(1);
  k_adam<<<(NW + 255) / 256, 256, 0, st>>>(w, g, m, v, NW, lr, b1, b2, 1e-8f, 1.f - std::pow(b1, (float)step),
                                           1.f - std::pow(b2, (float)step));
}

void sample(int64_t* idx, int batch, int64_t n, unsigned long long seed, unsigned long long step, cudaStream_t st) {
  count_launches(1);
  k_sample<<<(batch + 255) / 256, 256, 0, st>>>(idx, batch, n, seed, step);
}

// first feature: x0 (a start's doubles, [i][j][a][b]) when given, else t_MP2 = -(ia|jb)/D
__global__ void k_features(const double* __restrict__ gov, const double* __restrict__ eps, int o, int v,
                           const double* __restrict__ x0, float* X) {
  const int64_t n = (int64_t)o * o * v * v;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % v);
    int64_t r = e / v;
    const int a = (int)(r % v);
    r /= v;
    const int j = (int)(r % o), i = (int)(r / o);
    const double g = gov[(((int64_t)i * v + a) * o + j) * v + b];  // (ia|jb)
    const double D = eps[o + a] + eps[o + b] - eps[i] - eps[j];
    X[e * 3 + 0] = (float)(x0 ? x0[e] : -g / D);
    X[e * 3 + 1] = (float)D;
    X[e * 3 + 2] = (float)fabs(g);
  }
}

// T[e] = x[e] - X[e][0]: the correction a model is trained to predict
__global__ void k_targets(const double* __restrict__ x, const float* __restrict__ X, int64_t n, float* T) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    T[e] = (float)(x[e] - (double)X[e * 3]);
}

__global__ void k_add_delta(double* t2, const float* delta, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    t2[e] += (double)delta[e];
}

void features(const double* gov, const double* eps, int o, int v, float* X, cudaStream_t st, const double* x0) {
  const int64_t n = (int64_t)o * o * v * v;
  count_launches(1);
  k_features<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(gov, eps, o, v, x0, X);
}

__global__ void k_mp2_doubles(const double* __restrict__ gov, const double* __restrict__ eps, int o, int v,
                              double* __restrict__ t2) {
  const int64_t n = (int64_t)o * o * v * v;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % v);
    int64_t r = e / v;
    const int a = (int)(r % v);
    r /= v;
    const int j = (int)(r % o), i = (int)(r / o);
    t2[e] = -gov[(((int64_t)i * v + a) * o + j) * v + b] / (eps[o + a] + eps[o + b] - eps[i] - eps[j]);
  }
}

void mp2_doubles(const double* gov, const double* eps, int o, int v, double* t2, cudaStream_t st) {
  const int64_t n = (int64_t)o * o * v * v;
  count_launches(1);
  k_mp2_doubles<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(gov, eps, o, v, t2);
}

void targets(const double* x, const float* X, int64_t n, float* T, cudaStream_t st) {
  count_launches(1);
  k_targets<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(x, X, n, T);
}

void add_delta(double* t2, const float* delta, int64_t n, cudaStream_t st) {
  count_launches(1);
  k_add_delta<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(t2, delta, n);
}

// Deterministic initial weights (uniform, Glorot scale) from a host-side splitmix64 stream.
void init_weights(float* host_model, unsigned long long seed) {
  unsigned long long s = seed;
  auto next = [&]() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
  };
  auto fill = [&](int off, int count, double bound) {
    for (int i = 0; i < count; ++i) host_model[off + i] = (float)((2.0 * next() - 1.0) * bound);
  };
  fill(OW1, H * 3, std::sqrt(6.0 / (3 + H)));
  fill(OB1, H, 0.0);
  fill(OW2, H * H, std::sqrt(6.0 / (H + H)));
  fill(OB2, H, 0.0);
  fill(OW3, H, std::sqrt(6.0 / (H + 1)));
  host_model[OB3] = 0.f;
}

}  // namespace mlp
}  // namespace ccsd
