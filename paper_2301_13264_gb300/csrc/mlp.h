// Learned doubles guess: MLP kernels (mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ccsd {
namespace mlp {

constexpr int kParams = 128 * 3 + 128 + 128 * 128 + 128 + 128 + 1 + 7;  // weights + normalisation
constexpr int kTrainable = kParams - 7;

// out[r] = prediction for raw features X[r][3] (bf16-rounded weights, FP32 accumulation)
void predict(const float* model, const float* X, int64_t n, float* out, cudaStream_t st);
// grad[kTrainable] = d/dw of mean squared error over rows idx[0..n) (all rows if idx == nullptr),
// loss[0] = that error, in normalised target units
void gradient(const float* model, const float* X, const float* T, const int64_t* idx, int64_t n, float* grad,
              float* loss, cudaStream_t st);
void adam(float* w, const float* g, float* m, float* v, float lr, int step, cudaStream_t st);
void sample(int64_t* idx, int batch, int64_t n, unsigned long long seed, unsigned long long step, cudaStream_t st);
void init_weights(float* host_model, unsigned long long seed);
// X[(ijab)][3] = (x0, D, |(ia|jb)|) from the bare (kc|ld) block and orbital energies, with
// x0 the given start's doubles, or t_MP2 = -(ia|jb)/D when x0 is null
void features(const double* gov, const double* eps, int o, int v, float* X, cudaStream_t st,
              const double* x0 = nullptr);
// T[e] = x[e] - X[e][0] over n doubles: the correction from the start to the converged x
void targets(const double* x, const float* X, int64_t n, float* T, cudaStream_t st);
// t2[(ijab)] = -(ia|jb)/D, the first-order doubles, in FP64
void mp2_doubles(const double* gov, const double* eps, int o, int v, double* t2, cudaStream_t st);
// t2 += delta (float) over the o^2 v^2 doubles
void add_delta(double* t2, const float* delta, int64_t n, cudaStream_t st);

}  // namespace mlp
}  // namespace ccsd
