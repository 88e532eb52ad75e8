// Tensor-core (tcgen05) contraction path for the mixed-precision mode.
#include "exec.h"

namespace ccsd {

struct Executor::CacheEntry {
  const double* src = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
};

void Executor::clear_cache() {
  for (CacheEntry* e : cache_) {
    if (e->dev) cudaFree(e->dev);
    delete e;
  }
  cache_.clear();
  cache_bytes_ = 0;
}

bool Executor::tc_contract(int, int, int, int, const double*, int64_t, int64_t, int64_t, const double*, int64_t,
                           int64_t, int64_t, double*, int64_t, int64_t, int64_t, double, bool) {
  return false;
}

}  // namespace ccsd
