// Device memory for the library: the caller's allocator callbacks when the handle
// has them (ccsd_options.alloc / free / alloc_ctx), else the CUDA runtime.
//
// Every device allocation the library makes goes through dev_alloc / dev_free.
// The allocator in effect is the one of the handle whose C call is running on
// this thread (an AllocatorScope set up by the call); with none, the CUDA
// runtime is used exactly as before: cudaMallocAsync / cudaFreeAsync on the
// given stream for stream-ordered temporaries, cudaMalloc / cudaFree otherwise.
//
// Callback contract (stated in include/ccsd.h): alloc(bytes, stream, ctx)
// returns device memory of the handle's GPU that work queued on `stream` after
// the call may use, or NULL when it cannot (the library then returns
// CCSD_ERR_OOM); free(p, stream, ctx) releases it once the work already queued
// on `stream` has finished (the cudaFreeAsync ordering).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <stdexcept>
#include <string>
#include <vector>

namespace ccsd {

struct DeviceAllocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx) = nullptr;
  void (*free)(void* p, void* stream, void* ctx) = nullptr;
  void* ctx = nullptr;
  bool custom() const { return alloc != nullptr; }
};

// A device allocation failed (the callback returned NULL or the runtime ran out of memory).
struct OutOfMemory : std::runtime_error {
  explicit OutOfMemory(const std::string& m) : std::runtime_error(m) {}
};

// The allocator of the handle whose call runs on this thread (nullptr: the CUDA runtime),
// and that handle's stream (0 outside a handle's call).
const DeviceAllocator* active_allocator();
cudaStream_t active_stream();

// Makes `a` (with the handle's stream `st`) the active allocator of this thread for the
// scope's lifetime; the previous one is restored at the end of the scope.
class AllocatorScope {
 public:
  AllocatorScope(const DeviceAllocator* a, cudaStream_t st);
  ~AllocatorScope();
  AllocatorScope(const AllocatorScope&) = delete;
  AllocatorScope& operator=(const AllocatorScope&) = delete;

 private:
  const DeviceAllocator* prev_;
  cudaStream_t prev_st_;
};

// The stream-ordered allocations made while a library call runs: those still live when
// the call ends by an exception are released then, so that a failed call (an allocation
// refused half-way, a timed-out kernel) leaks nothing.  Allocations that outlive the call
// on purpose (cache entries) are taken out with dev_keep.
class TempScope {
 public:
  TempScope();
  ~TempScope();
  TempScope(const TempScope&) = delete;
  TempScope& operator=(const TempScope&) = delete;

 private:
  friend void* dev_alloc(size_t, cudaStream_t, bool);
  friend void dev_free(void*, cudaStream_t, bool);
  friend void dev_keep(void*);
  struct Rec {
    void* p;
    cudaStream_t st;
  };
  TempScope* prev_;
  int uncaught_;
  std::vector<Rec> live_;
};

// The stream-ordered allocation p outlives the current call (the TempScope forgets it).
void dev_keep(void* p);

// `bytes` of device memory usable by work queued on `st` from now on.  stream_ordered
// selects cudaMallocAsync (true) or cudaMalloc (false) when no callback is active.
// Throws OutOfMemory on failure; zero bytes allocate one byte.
void* dev_alloc(size_t bytes, cudaStream_t st, bool stream_ordered);
// Releases memory from dev_alloc with the same stream_ordered choice, after the work
// already queued on `st`.  Null is ignored.
void dev_free(void* p, cudaStream_t st, bool stream_ordered);

}  // namespace ccsd
