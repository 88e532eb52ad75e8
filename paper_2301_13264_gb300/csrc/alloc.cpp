// Device memory through the caller's allocator callbacks or the CUDA runtime (alloc.h).
#include "alloc.h"

#include <exception>

namespace ccsd {

namespace {
thread_local const DeviceAllocator* tl_allocator = nullptr;
thread_local cudaStream_t tl_stream = nullptr;
thread_local TempScope* tl_temps = nullptr;
}  // namespace

TempScope::TempScope() : prev_(tl_temps), uncaught_(std::uncaught_exceptions()) { tl_temps = this; }

TempScope::~TempScope() {
  tl_temps = prev_;
  if (std::uncaught_exceptions() > uncaught_) {
    for (const Rec& r : live_) dev_free(r.p, r.st, true);
  } else if (prev_) {
    // still live at a normal end: the enclosing call owns them now
    prev_->live_.insert(prev_->live_.end(), live_.begin(), live_.end());
  }
}

void dev_keep(void* p) {
  if (!tl_temps || !p) return;
  auto& v = tl_temps->live_;
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i].p == p) {
      v.erase(v.begin() + i);
      return;
    }
}

const DeviceAllocator* active_allocator() { return tl_allocator; }
cudaStream_t active_stream() { return tl_stream; }

AllocatorScope::AllocatorScope(const DeviceAllocator* a, cudaStream_t st) : prev_(tl_allocator), prev_st_(tl_stream) {
  tl_allocator = (a && a->custom()) ? a : nullptr;
  tl_stream = st;
}

AllocatorScope::~AllocatorScope() {
  tl_allocator = prev_;
  tl_stream = prev_st_;
}

void* dev_alloc(size_t bytes, cudaStream_t st, bool stream_ordered) {
  if (bytes == 0) bytes = 1;
  const DeviceAllocator* a = tl_allocator;
  void* p = nullptr;
  if (a) {
    p = a->alloc(bytes, (void*)st, a->ctx);
    if (!p) throw OutOfMemory("device allocation of " + std::to_string(bytes) + " bytes refused by the allocator");
  } else {
    const cudaError_t e = stream_ordered ? cudaMallocAsync(&p, bytes, st) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();  // a failed allocation leaves no sticky error
      throw OutOfMemory("device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
  }
  if (stream_ordered && tl_temps) tl_temps->live_.push_back(TempScope::Rec{p, st});
  return p;
}

void dev_free(void* p, cudaStream_t st, bool stream_ordered) {
  if (!p) return;
  if (stream_ordered && tl_temps) {
    auto& v = tl_temps->live_;
    for (size_t i = v.size(); i-- > 0;)
      if (v[i].p == p) {
        v.erase(v.begin() + i);
        break;
      }
  }
  const DeviceAllocator* a = tl_allocator;
  if (a) {
    if (a->free) a->free(p, (void*)st, a->ctx);
    return;
  }
  if (stream_ordered)
    cudaFreeAsync(p, st);
  else
    cudaFree(p);
}

}  // namespace ccsd
