// Allocation-free derivative couplings from densities already held by a handle.
//
// Some callers cannot allocate device memory at the point where they need the
// coupling: a dynamics driver that runs inside a memory pool owned by another
// framework (which may be full, or may forbid foreign cudaMalloc calls), or
// code that must not hit the allocator between time steps because an
// allocation can synchronise the device and stall the trajectory.  For them
// this file provides ccsd_derivative_coupling_noalloc, which contracts the
// held densities with caller-provided device directions using a fixed scratch
// array that lives in this library's device image.
//
// The scratch is a file-scope __device__ array of kScratch doubles (16 KiB).
// Every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address, so the address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, and cached here.  The device is the handle's (the one current when
// the handle was created), not whichever device is current at the call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ccsd.h"
#include "kernels.cuh"

namespace ccsd {
bool held_densities(ccsd_handle c, int k, int l, const double** D, const double** Z, int* n, int* naux,
                    cudaStream_t* st, int* device);
void set_error(ccsd_handle c, const char* msg);
}  // namespace ccsd

namespace {

constexpr int kScratch = 2048;          // doubles
constexpr int kPartials = 1024;         // reduction partials (launch_dot uses 512)
constexpr int kMaxDirections = 256;     // results: three slots per direction after the partials
static_assert(kPartials + 3 * kMaxDirections <= kScratch, "scratch too small");

__device__ __align__(256) double g_coupling_scratch[kScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on GPU `dev`, which must be current (looked up
// once per device and cached).
double* scratch_for_device(int dev, cudaError_t* err) {
  *err = cudaSuccess;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_coupling_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

__global__ void k_add_parts(int ndir, const double* h_part, const double* b_part, double* out) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < ndir) out[d] = h_part[d] + b_part[d];
}

// true when p is device (or managed) memory of GPU `dev`: the kernels below read it
// from the handle's device and no peer access is set up
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Makes GPU `dev` current for the guard's lifetime (the handle's stream belongs to it)
// and restores the caller's device afterwards.  Allocates nothing.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    if (err != cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" ccsd_status ccsd_derivative_coupling_noalloc(ccsd_handle h, int k, int l, int ndir, const double* dh,
                                                        const double* dB, double* F) {
  using namespace ccsd;
  if (!h) return CCSD_ERR_ARG;
  if (ndir < 1 || ndir > kMaxDirections || !dh || !dB || !F) {
    set_error(h, "noalloc coupling: need 1 <= ndir <= 256 and non-null dh, dB, F");
    return CCSD_ERR_ARG;
  }
  const double *D = nullptr, *Z = nullptr;
  int n = 0, naux = 0;
  cudaStream_t st = 0;
  int dev = 0;
  if (!held_densities(h, k, l, &D, &Z, &n, &naux, &st, &dev)) {
    set_error(h, "noalloc coupling: call ccsd_coupling_densities for this (k, l) first");
    return CCSD_ERR_STATE;
  }
  DeviceGuard on_handle_device(dev);
  if (on_handle_device.err != cudaSuccess) {
    set_error(h, cudaGetErrorString(on_handle_device.err));
    return CCSD_ERR_CUDA;
  }
  if (!on_device(dh, dev) || !on_device(dB, dev)) {
    set_error(h, "noalloc coupling: dh and dB must be device memory of the handle's GPU");
    return CCSD_ERR_ARG;
  }
  cudaError_t err = cudaSuccess;
  double* s = scratch_for_device(dev, &err);
  if (!s) {
    set_error(h, cudaGetErrorString(err));
    return CCSD_ERR_CUDA;
  }
  double* partials = s;
  double* h_part = s + kPartials;
  double* b_part = h_part + kMaxDirections;
  double* sum = b_part + kMaxDirections;
  const long long nn = (long long)n * n, nb = (long long)naux * nn;
  // every slot used below is written before it is read, so nothing is cleared;
  // launch_dot counts its own two launches, so the call launches 4 * ndir + 1 kernels
  for (int d = 0; d < ndir; ++d) {
    launch_dot(nn, D, dh + d * nn, h_part + d, partials, st);
    launch_dot(nb, Z, dB + d * nb, b_part + d, partials, st);
  }
  count_launches(1);
  k_add_parts<<<(ndir + 127) / 128, 128, 0, st>>>(ndir, h_part, b_part, sum);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(F, sum, ndir * sizeof(double), cudaMemcpyDefault, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    set_error(h, cudaGetErrorString(err));
    return CCSD_ERR_CUDA;
  }
  return CCSD_OK;
}
