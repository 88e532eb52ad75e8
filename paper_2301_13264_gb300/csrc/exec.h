// Executes tensor programs on one GPU stream.
//
// Each contraction out[lo] += alpha * sum a[la] b[lb] is mapped onto one
// batched GEMM: labels shared by a, b and out are the batch, labels of a and
// out the M extent, of b and out the N extent, of a and b the K extent.
// Operands whose memory already has that shape are addressed in place;
// others are gathered into a contiguous buffer first.  Temporaries of a
// program run are allocated and freed stream-ordered around their live range.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

#include "ir.h"
#include "kernels.cuh"

namespace ccsd {

// PREC_FP64_TC: FP64-grade contractions on the tensor cores (fixed-point bf16 slices,
// exact per-chunk sums; fp64_tc.cu) for contractions above tc_min_flops, FP64 DFMA below
enum Precision : int { PREC_FP64 = 0, PREC_MIXED = 1, PREC_FP64_TC = 2 };

struct ExecStats {
  int64_t gemm_calls = 0, tc_calls = 0, packs = 0, scatters = 0, axpys = 0, ladders = 0;
  double gemm_flops = 0.0, tc_flops = 0.0;
};

class Executor {
 public:
  Executor(const Graph& g, int o, int v, int naux, int nvec_max, cudaStream_t st);
  ~Executor();
  Executor(const Executor&) = delete;
  Executor& operator=(const Executor&) = delete;

  void set_nvec(int nvec);
  int nvec() const { return nvec_; }
  // bind an external device buffer; zstride is the distance between vector slices
  // of a tensor whose leading class is 'z' (-1: contiguous)
  void bind(int t, double* p, int64_t zstride = -1);
  void unbind(int t);
  // allocate an owned buffer that persists across program runs
  void alloc_persistent(int t);
  double* ptr(int t) const { return ts_[t].p; }
  int64_t numel(int t) const;  // with the current nvec
  void run(const Prog& p);

  void set_precision(int prec, int splits) {
    prec_ = prec;
    splits_ = splits;
  }
  int precision() const { return prec_; }
  void set_stream(cudaStream_t st) { st_ = st; }
  // While a run is captured into a CUDA graph it must not synchronise: the error
  // flag of the tensor-core kernels is then read after the graph has run.
  bool capturing = false;
  // tensor-core tile choice: 0 = by output width, 1 = time the candidate tile
  // widths and split counts once per GEMM shape and keep the fastest
  int autotune = 0;
  // contractions with fewer flops than this stay on the FP64 path in mixed mode
  double tc_min_flops = 1.0e8;
  // clock cycles a pipeline wait of a tensor-core kernel may take before the kernel
  // raises the error flag and exits (0: the default bound, about 2 s)
  long long wait_cycles = 0;
  // failure injection for tests: the next tensor-core GEMM launch issues no operand
  // loads, so its waits run out after wait_cycles (cleared by that launch)
  bool stall_next = false;
  ExecStats stats;
  cudaStream_t stream() const { return st_; }
  // device scratch for reductions
  double* scratch(int64_t n);
  // size of the largest bf16 operand cache entry, for tests
  size_t cache_bytes() const { return cache_bytes_; }
  void clear_cache();

 private:
  struct TS {
    double* p = nullptr;
    bool owned = false;
    bool bound = false;
    int64_t zstride = -1;
  };
  struct SView {
    double* base;
    int nd;
    int64_t ext[kMaxDims], str[kMaxDims];
  };
  struct Lab {
    char c;
    int64_t e, s;
  };
  SView resolve(const Ref& r) const;
  int64_t extent(char cls) const;
  std::vector<Lab> merge(const SView& v, const std::string& lab) const;
  void zero_tensor(int t);
  void exec_contract(const Op& op);
  void exec_axpy(const Op& op);
  double* tmp_alloc(int64_t n);
  void tmp_free(double* p);

  const Graph& g_;
  int o_, v_, naux_, nvec_max_, nvec_;
  cudaStream_t st_;
  std::vector<TS> ts_;
  int prec_ = PREC_FP64, splits_ = 3;
  double* scratch_ = nullptr;
  int64_t scratch_n_ = 0;
  size_t cache_bytes_ = 0;

  int* tc_err_ = nullptr;  // device flag raised by a tensor-core kernel whose wait timed out
  struct ProfRec {
    cudaEvent_t a, b;
    double flops, issued;
    bool tc;
    bool ladder = false;
    int engine = 0;  // 0 FP64 DFMA, 1 split-bf16 tensor cores, 2 FP64-grade tensor cores
    int64_t batch = 1, m = 0, n = 0, k = 0;
    std::string label;
  };
  // the contraction an op performs, as out[labels] += a[labels] * b[labels]
  std::string op_label(const Op& op) const;
  bool profiling_ = false;
  std::vector<ProfRec> prof_;

 public:
  // tensor-core path (tc_gemm.cu); returns false when the op is not eligible.
  // C = alpha * A B^T + beta * C with beta in {0, 1}.  A and B are strided
  // gathers over (row dims..., K dims...) with source strides in s1; constant
  // operands keep their bf16 slices cached for the life of the executor.
  // With om/on given, element (m, n) is written at C + off(m; om) + off(n; on) (row-major
  // decomposition over ext, strides in s0) instead of C + m*sCm + n*sCn.
  bool tc_contract(int M, int N, int K, const double* A, const Strided& Ag, const double* B, const Strided& Bg,
                   double* C, int64_t sCm, int64_t sCn, double alpha, double beta, bool a_const, bool b_const,
                   const Strided* om = nullptr, const Strided* on = nullptr);
  // the same contraction through the FP64-grade tensor-core products (fp64_tc.cu);
  // constant operands keep their fixed-point slices cached like the split slices
  bool fp64tc_contract(int M, int N, int K, const double* A, const Strided& Ag, const double* B, const Strided& Bg,
                       double* C, int64_t sCm, int64_t sCn, double alpha, double beta, bool a_const, bool b_const,
                       const Strided* om = nullptr, const Strided* on = nullptr);
  // tcgen05 GEMM on prepared bf16 slices: a [S][Mp][Kp], b [S][Np][Kp] (rows and K
  // zero-padded; Mp a multiple of 128, Np of the tile width chosen for N);
  // C[m*sCm + n*sCn] = alpha * sum + beta * C.
  // BN (tile width, 0: by N) and nsplit (split-K count, 0: heuristic) may be given.
  void tc_run(const void* a, int64_t Mp, const void* b, int64_t Np, int K, int64_t Kp, int S, int M, int N, double* C,
              int64_t sCm, int64_t sCn, double alpha, double beta, const Strided* om = nullptr,
              const Strided* on = nullptr, int BN = 0, int nsplit = 0);
  struct TcChoice {
    int bn, nsplit;  // nsplit 0: heuristic
  };
  // tile width and split count for a tensor-core GEMM shape (timed once per shape when autotune is on)
  TcChoice tc_choice(int M, int N, int64_t Kp, int S, bool strided);
  std::map<std::array<int64_t, 4>, TcChoice> tc_tuned_;
  // pp-ladder contractions against the bare vvvv tensor (ladder.cu); false if op is not one
  bool try_ladder(const Op& op);
  int ladder_w_ = -1;  // tensor id of W[a][b][c][d] = (ac|bd)
  const int2* pair_table();
  struct WPM {
    bool mixed = false;
    int S = 0;
    void *plus = nullptr, *minus = nullptr;
    int64_t rows_p = 0, ld = 0;
    size_t bytes = 0;
  };
  std::vector<WPM> wpm_;
  void* pairs_ = nullptr;
  struct LadderTables {
    std::vector<int64_t> offA, offIJ, offJI;
    std::vector<unsigned char> same;
    void* dev;
  };
  std::vector<LadderTables> ladder_tables_;
  // value of the device error flag (synchronises the stream); 0 when no tensor-core kernel ran
  int tc_error();
  // tensors whose values never change after set-up (their bf16 slices may be cached)
  std::set<int> const_tensors;
  // tensors that change only with the amplitudes (the primal intermediates and the
  // amplitudes themselves): their bf16 slices are kept across runs of the derivative
  // programs, which leave them unchanged, until invalidate_frozen() is called because
  // the amplitudes changed
  std::set<int> frozen_tensors;
  void invalidate_frozen();
  // changes whenever cached operand slices are dropped (graphs that captured their
  // addresses must then be captured again)
  uint64_t cache_epoch() const { return cache_epoch_; }
  // Profiling: when on, every GEMM launch is bracketed by CUDA events on the
  // executor's stream; collect() returns per-engine totals and clears the records.
  struct ProfTotals {
    long long tc_launches = 0, fp64_launches = 0;
    double tc_ms = 0, tc_flops = 0, tc_issued = 0, fp64_ms = 0, fp64_flops = 0;
    double top_ms = 0, top_flops = 0, top_issued = 0;  // the largest tensor-core contraction
    long long top_launches = 0;
    double ladder_ms = 0, ladder_flops = 0, ladder_issued = 0;  // pp-ladder GEMMs
    long long ladder_launches = 0;
  };
  void profile(bool on);
  ProfTotals collect();
  // one line per GEMM launch of the last collect(), in launch order
  struct ProfLine {
    std::string label;
    int engine;
    bool ladder;
    int64_t batch, m, n, k;
    double ms, flops, issued;
  };
  const std::vector<ProfLine>& profile_lines() const { return prof_lines_; }
  std::vector<ProfLine> prof_lines_;
  double last_tc_issued = 0.0;  // MMA flops of the last tensor-core launch (padding included)
  struct CacheEntry;
  std::vector<CacheEntry*> cache_;

 private:
  bool frozen_run_ = false;  // the current run writes amplitude-dependent tensors
  uint64_t cache_epoch_ = 0;
  void drop_cache_range(const double* p, int64_t n);
};

// A device-side wait exceeded its budget (the kernel raised its error flag).
struct DeviceTimeout : std::runtime_error {
  explicit DeviceTimeout(const std::string& m) : std::runtime_error(m) {}
};

}  // namespace ccsd
