// Program executor: label analysis, operand gathering, GEMM dispatch.
#include "exec.h"

#include "alloc.h"

#include <algorithm>
#include <map>
#include <cstdio>
#include <cstdlib>
#include <exception>
#include <stdexcept>

namespace ccsd {

#define CK(x)                                                                                   \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) throw std::runtime_error(std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

Executor::Executor(const Graph& g, int o, int v, int naux, int nvec_max, cudaStream_t st)
    : g_(g), o_(o), v_(v), naux_(naux), nvec_max_(nvec_max), nvec_(1), st_(st) {
  ts_.resize(g.T.size());
}

Executor::~Executor() {
  clear_cache();
  for (auto& t : ts_)
    if (t.owned && t.p) dev_free(t.p, st_, false);
  dev_free(scratch_, st_, false);
}

void Executor::set_nvec(int nvec) {
  if (nvec < 1 || nvec > nvec_max_) throw std::runtime_error("nvec out of range");
  nvec_ = nvec;
}

int64_t Executor::extent(char c) const {
  switch (c) {
    case 'o': return o_;
    case 'v': return v_;
    case 'n': return o_ + v_;
    case 'x': return naux_;
    case 'z': return nvec_;
  }
  throw std::runtime_error(std::string("bad class ") + c);
}

int64_t Executor::numel(int t) const {
  int64_t n = 1;
  for (char c : g_.T[t].cls) n *= extent(c);
  return n;
}

void Executor::bind(int t, double* p, int64_t zstride) {
  TS& s = ts_[t];
  if (s.owned && s.p) dev_free(s.p, st_, false);
  s.p = p;
  s.owned = false;
  s.bound = true;
  s.zstride = zstride;
}

void Executor::unbind(int t) {
  TS& s = ts_[t];
  if (s.bound) {
    s.p = nullptr;
    s.bound = false;
    s.zstride = -1;
  }
}

void Executor::alloc_persistent(int t) {
  TS& s = ts_[t];
  if (s.p) return;
  int64_t n = 1;
  for (char c : g_.T[t].cls) n *= (c == 'z') ? nvec_max_ : extent(c);
  s.p = (double*)dev_alloc(std::max<int64_t>(n, 1) * sizeof(double), st_, false);
  CK(cudaMemsetAsync(s.p, 0, std::max<int64_t>(n, 1) * sizeof(double), st_));
  s.owned = true;
}

double* Executor::scratch(int64_t n) {
  if (n > scratch_n_) {
    dev_free(scratch_, st_, false);
    scratch_ = nullptr;
    scratch_ = (double*)dev_alloc(n * sizeof(double), st_, false);
    scratch_n_ = n;
  }
  return scratch_;
}

double* Executor::tmp_alloc(int64_t n) {
  return (double*)dev_alloc(std::max<int64_t>(n, 1) * sizeof(double), st_, true);
}

void Executor::tmp_free(double* p) {
  dev_free(p, st_, true);
}

Executor::SView Executor::resolve(const Ref& r) const {
  const std::string& cls = g_.T[r.t].cls;
  const TS& s = ts_[r.t];
  if (!s.p) throw std::runtime_error("tensor without storage: " + g_.T[r.t].name);
  SView v;
  v.nd = (int)cls.size();
  if (v.nd > kMaxDims) throw std::runtime_error("too many dims");
  if ((int)r.blk.size() != v.nd) throw std::runtime_error("block spec mismatch for " + g_.T[r.t].name);
  int64_t full[kMaxDims];
  for (int d = 0; d < v.nd; ++d) full[d] = extent(cls[d]);
  if (v.nd > 0) {
    v.str[v.nd - 1] = 1;
    for (int d = v.nd - 2; d >= 0; --d) v.str[d] = v.str[d + 1] * full[d + 1];
    if (cls[0] == 'z' && s.zstride >= 0) v.str[0] = s.zstride;
  }
  int64_t off = 0;
  for (int d = 0; d < v.nd; ++d) {
    v.ext[d] = full[d];
    if (cls[d] == 'n') {
      if (r.blk[d] == 'o') {
        v.ext[d] = o_;
      } else if (r.blk[d] == 'v') {
        v.ext[d] = v_;
        off += (int64_t)o_ * v.str[d];
      }
    }
  }
  v.base = s.p + off;
  return v;
}

std::vector<Executor::Lab> Executor::merge(const SView& v, const std::string& lab) const {
  if ((int)lab.size() != v.nd) throw std::runtime_error("label count mismatch");
  std::vector<Lab> out;
  for (int d = 0; d < v.nd; ++d) {
    bool found = false;
    for (auto& l : out)
      if (l.c == lab[d]) {
        if (l.e != v.ext[d]) throw std::runtime_error("diagonal extent mismatch");
        l.s += v.str[d];
        found = true;
      }
    if (!found) out.push_back(Lab{lab[d], v.ext[d], v.str[d]});
  }
  return out;
}

void Executor::zero_tensor(int t) {
  const std::string& cls = g_.T[t].cls;
  const TS& s = ts_[t];
  int64_t n = numel(t);
  bool contig = !(cls.size() > 0 && cls[0] == 'z' && s.zstride >= 0 && s.zstride != n / nvec_);
  if (contig) {
    CK(cudaMemsetAsync(s.p, 0, std::max<int64_t>(n, 1) * sizeof(double), st_));
    return;
  }
  Strided sp;
  sp.ndim = 2;
  sp.ext[0] = nvec_;
  sp.ext[1] = n / nvec_;
  sp.s0[0] = s.zstride;
  sp.s0[1] = 1;
  sp.s1[0] = sp.s1[1] = 0;
  launch_zero_strided(s.p, sp, st_);
}

static bool has(const std::vector<char>& v, char c) { return std::find(v.begin(), v.end(), c) != v.end(); }

// Collapse a group of labels (in the given order) of a view into one stride.
static bool collapse(const std::vector<char>& group, const std::map<char, std::pair<int64_t, int64_t>>& es,
                     int64_t& stride) {
  if (group.empty()) {
    stride = 0;
    return true;
  }
  // drop extent-1 labels: they do not constrain the layout
  std::vector<std::pair<int64_t, int64_t>> g;
  for (char c : group) {
    auto& p = es.at(c);
    if (p.first != 1) g.push_back(p);
  }
  if (g.empty()) {
    stride = 0;
    return true;
  }
  for (size_t i = 0; i + 1 < g.size(); ++i)
    if (g[i].second != g[i + 1].second * g[i + 1].first) return false;
  stride = g.back().second;
  return true;
}

void Executor::exec_contract(const Op& op) {
  if (try_ladder(op)) return;
  SView O = resolve(op.out), A = resolve(op.a), B = resolve(op.b);
  auto lo = merge(O, op.lo), la = merge(A, op.la), lb = merge(B, op.lb);
  std::map<char, std::pair<int64_t, int64_t>> eo, ea, eb;
  std::vector<char> co, ca, cb;
  for (auto& l : lo) {
    eo[l.c] = {l.e, l.s};
    co.push_back(l.c);
  }
  for (auto& l : la) {
    ea[l.c] = {l.e, l.s};
    ca.push_back(l.c);
  }
  for (auto& l : lb) {
    eb[l.c] = {l.e, l.s};
    cb.push_back(l.c);
  }
  std::vector<char> bat, Ml, Nl, Kl;
  for (char c : co) {
    bool ia = has(ca, c), ib = has(cb, c);
    if (ia && ib)
      bat.push_back(c);
    else if (ia)
      Ml.push_back(c);
    else if (ib)
      Nl.push_back(c);
    else
      throw std::runtime_error("output label not in operands");
  }
  for (char c : ca)
    if (!has(co, c)) {
      if (!has(cb, c)) throw std::runtime_error("label summed over one operand");
      Kl.push_back(c);
    }
  for (char c : cb)
    if (!has(co, c) && !has(ca, c)) throw std::runtime_error("label summed over one operand");
  auto ext_of = [&](char c) -> int64_t {
    int64_t e = eo.count(c) ? eo[c].first : ea.count(c) ? ea[c].first : eb[c].first;
    if ((eo.count(c) && eo[c].first != e) || (ea.count(c) && ea[c].first != e) || (eb.count(c) && eb[c].first != e))
      throw std::runtime_error("label extent mismatch");
    return e;
  };
  int64_t Bt = 1, M = 1, N = 1, K = 1;
  for (char c : bat) Bt *= ext_of(c);
  for (char c : Ml) M *= ext_of(c);
  for (char c : Nl) N *= ext_of(c);
  for (char c : Kl) K *= ext_of(c);
  if (Bt == 0 || M == 0 || N == 0) return;
  if (K == 0) return;
  if (Bt > 65535 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) throw std::runtime_error("GEMM too large");
  const double flops = 2.0 * (double)Bt * M * N * K;

  // output addressing: direct when the out view has the [bat][M][N] shape
  int64_t sCb, sCm, sCn;
  const bool cdirect = collapse(bat, eo, sCb) && collapse(Ml, eo, sCm) && collapse(Nl, eo, sCn);
  auto scatter_from = [&](const double* Ctmp) {
    Strided sp;
    std::vector<char> order = bat;
    order.insert(order.end(), Ml.begin(), Ml.end());
    order.insert(order.end(), Nl.begin(), Nl.end());
    sp.ndim = (int)order.size();
    int64_t st = 1;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      sp.ext[d] = eo[order[d]].first;
      sp.s0[d] = eo[order[d]].second;
      sp.s1[d] = st;
      st *= sp.ext[d];
    }
    launch_axpy_strided(O.base, Ctmp, sp, op.alpha, st_);
    stats.scatters++;
  };

  // tensor-core path: operands are gathered straight from their strided FP64
  // layout into bf16 slices (no FP64 staging copy)
  // tensor cores: large enough, and not mostly padding (the MMA tile pads the longer side to
  // 128 rows, the shorter to 64 and K to 64: a rank-1 update or a dot product of two huge vectors
  // would issue hundreds of times its work and slice operands of tens of GB)
  auto pad = [](int64_t x, int64_t q) { return (x + q - 1) / q * q; };
  const double padded = (double)pad(std::max(M, N), 128) * (double)pad(std::min(M, N), 64) * (double)pad(K, 64);
  const bool tc_shape = padded <= 16.0 * (double)M * (double)N * (double)K;
  if ((prec_ == PREC_MIXED || prec_ == PREC_FP64_TC) && flops >= tc_min_flops && Bt == 1 && tc_shape) {
    auto gather = [&](std::map<char, std::pair<int64_t, int64_t>>& es, const std::vector<char>& rows) {
      Strided g;
      std::vector<char> order = rows;
      order.insert(order.end(), Kl.begin(), Kl.end());
      g.ndim = (int)order.size();
      for (int d = 0; d < g.ndim; ++d) {
        g.ext[d] = es[order[d]].first;
        g.s1[d] = es[order[d]].second;
        g.s0[d] = 0;
      }
      return g;
    };
    // amplitude-dependent operands are cached only in runs that leave all of them unchanged
    // (the derivative programs), not in the forward program that recomputes them
    auto cacheable = [&](int t) { return const_tensors.count(t) > 0 || (frozen_tensors.count(t) > 0 && !frozen_run_); };
    const bool a_const = cacheable(op.a.t), b_const = cacheable(op.b.t);
    // The gather of an operand sliced anew at every call reads coalesced only if its last K
    // label or its last row label is contiguous in it.  When neither is but another row label
    // is, and the operand outweighs the output, that label goes last in the row order (the
    // output follows the same order through its offset table).
    std::vector<char> Mt = Ml, Nt = Nl;
    auto unit = [](std::map<char, std::pair<int64_t, int64_t>>& es, char c) {
      return es[c].first > 1 && (es[c].second == 1 || es[c].second == -1);
    };
    auto favor = [&](std::vector<char>& rows, std::map<char, std::pair<int64_t, int64_t>>& es, int64_t nrows,
                     bool cached) {
      if (cached || rows.size() < 2 || (double)nrows * K < 2.0 * (double)M * N) return false;
      if ((!Kl.empty() && unit(es, Kl.back())) || unit(es, rows.back())) return false;
      for (size_t i = 0; i + 1 < rows.size(); ++i)
        if (unit(es, rows[i])) {
          const char c = rows[i];
          rows.erase(rows.begin() + i);
          rows.push_back(c);
          return true;
        }
      return false;
    };
    const bool reordered_a = favor(Mt, ea, M, a_const);
    const bool reordered_b = favor(Nt, eb, N, b_const);
    const bool cdir = cdirect && !reordered_a && !reordered_b;
    Strided ag = gather(ea, Mt), bg = gather(eb, Nt);
    // non-contiguous outputs are addressed by the GEMM epilogue through the output's own strides
    Strided om, on;
    auto out_dims = [&](const std::vector<char>& labels, Strided& g) {
      g.ndim = (int)labels.size();
      for (int d = 0; d < g.ndim; ++d) {
        g.ext[d] = eo[labels[d]].first;
        g.s0[d] = eo[labels[d]].second;
        g.s1[d] = 0;
      }
      if (g.ndim == 0) {
        g.ndim = 1;
        g.ext[0] = 1;
        g.s0[0] = g.s1[0] = 0;
      }
    };
    if (!cdir) {
      out_dims(Mt, om);
      out_dims(Nt, on);
    }
    double* Ct = nullptr;
    ProfRec rec{};
    if (profiling_) {
      CK(cudaEventCreate(&rec.a));
      CK(cudaEventCreate(&rec.b));
      CK(cudaEventRecord(rec.a, st_));
      rec.flops = flops;
      rec.engine = prec_ == PREC_FP64_TC ? 2 : 1;
      rec.batch = Bt;
      rec.m = M;
      rec.n = N;
      rec.k = K;
      rec.label = op_label(op);
    }
    bool ok = tc_contract((int)M, (int)N, (int)K, A.base, ag, B.base, bg, O.base, cdir ? sCm : 0, cdir ? sCn : 0,
                          op.alpha, 1.0, a_const, b_const, cdir ? nullptr : &om, cdir ? nullptr : &on);
    if (profiling_) {
      CK(cudaEventRecord(rec.b, st_));
      rec.tc = ok;
      rec.issued = ok ? last_tc_issued : 0.0;
      if (ok)
        prof_.push_back(rec);
      else {
        cudaEventDestroy(rec.a);
        cudaEventDestroy(rec.b);
      }
    }
    if (ok) {
      stats.tc_calls++;
      stats.tc_flops += flops;
      return;
    }
    if (Ct) tmp_free(Ct);
  }

  // operand A: [bat][M][K]
  const double* Ap = A.base;
  int64_t sAb, sAm, sAk;
  double* Apack = nullptr;
  if (!(collapse(bat, ea, sAb) && collapse(Ml, ea, sAm) && collapse(Kl, ea, sAk))) {
    Apack = tmp_alloc(Bt * M * K);
    Strided sp;
    std::vector<char> order = bat;
    order.insert(order.end(), Ml.begin(), Ml.end());
    order.insert(order.end(), Kl.begin(), Kl.end());
    sp.ndim = (int)order.size();
    int64_t st = 1;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      sp.ext[d] = ea[order[d]].first;
      sp.s1[d] = ea[order[d]].second;
      sp.s0[d] = st;
      st *= sp.ext[d];
    }
    launch_copy_strided(Apack, A.base, sp, st_);
    stats.packs++;
    Ap = Apack;
    sAb = M * K;
    sAm = K;
    sAk = 1;
  }
  const double* Bp = B.base;
  int64_t sBb, sBn, sBk;
  double* Bpack = nullptr;
  if (!(collapse(bat, eb, sBb) && collapse(Nl, eb, sBn) && collapse(Kl, eb, sBk))) {
    Bpack = tmp_alloc(Bt * N * K);
    Strided sp;
    std::vector<char> order = bat;
    order.insert(order.end(), Nl.begin(), Nl.end());
    order.insert(order.end(), Kl.begin(), Kl.end());
    sp.ndim = (int)order.size();
    int64_t st = 1;
    for (int d = sp.ndim - 1; d >= 0; --d) {
      sp.ext[d] = eb[order[d]].first;
      sp.s1[d] = eb[order[d]].second;
      sp.s0[d] = st;
      st *= sp.ext[d];
    }
    launch_copy_strided(Bpack, B.base, sp, st_);
    stats.packs++;
    Bp = Bpack;
    sBb = N * K;
    sBn = K;
    sBk = 1;
  }
  double* Ctmp = nullptr;
  double* Cp = O.base;
  double alpha = op.alpha, beta = 1.0;
  if (!cdirect) {
    Ctmp = tmp_alloc(Bt * M * N);
    Cp = Ctmp;
    sCb = M * N;
    sCm = N;
    sCn = 1;
    alpha = 1.0;
    beta = 0.0;
  }
  ProfRec rec{};
  if (profiling_) {
    CK(cudaEventCreate(&rec.a));
    CK(cudaEventCreate(&rec.b));
    CK(cudaEventRecord(rec.a, st_));
    rec.flops = flops;
    rec.engine = 0;
    rec.batch = Bt;
    rec.m = M;
    rec.n = N;
    rec.k = K;
    rec.label = op_label(op);
  }
  GemmArgs ga;
  ga.batch = (int)Bt;
  ga.M = (int)M;
  ga.N = (int)N;
  ga.K = (int)K;
  ga.A = Ap;
  ga.sAb = sAb;
  ga.sAm = sAm;
  ga.sAk = sAk;
  ga.B = Bp;
  ga.sBb = sBb;
  ga.sBn = sBn;
  ga.sBk = sBk;
  ga.C = Cp;
  ga.sCb = sCb;
  ga.sCm = sCm;
  ga.sCn = sCn;
  ga.alpha = alpha;
  ga.beta = beta;
  launch_dgemm(ga, st_);
  stats.gemm_calls++;
  stats.gemm_flops += flops;
  if (profiling_) {
    CK(cudaEventRecord(rec.b, st_));
    rec.tc = false;
    rec.issued = flops;
    prof_.push_back(rec);
  }
  if (!cdirect) scatter_from(Ctmp);
  if (Apack) tmp_free(Apack);
  if (Bpack) tmp_free(Bpack);
  if (Ctmp) tmp_free(Ctmp);
}

void Executor::profile(bool on) {
  if (!on && !prof_.empty()) collect();  // records not yet collected (the last collect's lines stay)
  profiling_ = on;
}

std::string Executor::op_label(const Op& op) const {
  std::string s = g_.T[op.out.t].name + "[" + op.lo + "] += " + g_.T[op.a.t].name + "[" + op.la + "]";
  if (op.kind == 'C') s += " * " + g_.T[op.b.t].name + "[" + op.lb + "]";
  return s;
}

Executor::ProfTotals Executor::collect() {
  ProfTotals t;
  CK(cudaStreamSynchronize(st_));
  double top = 0.0;
  for (const ProfRec& r : prof_) if (r.tc) top = std::max(top, r.flops);
  prof_lines_.clear();
  prof_lines_.reserve(prof_.size());
  for (const ProfRec& r : prof_) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    prof_lines_.push_back(ProfLine{r.label, r.engine, r.ladder, r.batch, r.m, r.n, r.k, (double)ms, r.flops, r.issued});
    if (r.ladder) {
      t.ladder_launches++;
      t.ladder_ms += ms;
      t.ladder_flops += r.flops;
      t.ladder_issued += r.issued;
    }
    if (r.tc) {
      t.tc_launches++;
      t.tc_ms += ms;
      t.tc_flops += r.flops;
      t.tc_issued += r.issued;
      if (r.flops == top) {
        t.top_launches++;
        t.top_ms += ms;
        t.top_flops += r.flops;
        t.top_issued += r.issued;
      }
    } else {
      t.fp64_launches++;
      t.fp64_ms += ms;
      t.fp64_flops += r.flops;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  prof_.clear();
  return t;
}

void Executor::exec_axpy(const Op& op) {
  SView O = resolve(op.out), A = resolve(op.a);
  auto lo = merge(O, op.lo), la = merge(A, op.la);
  if (lo.size() != la.size()) throw std::runtime_error("axpy label sets differ");
  Strided sp;
  sp.ndim = (int)lo.size();
  for (int d = 0; d < sp.ndim; ++d) {
    sp.ext[d] = lo[d].e;
    sp.s0[d] = lo[d].s;
    bool found = false;
    for (auto& l : la)
      if (l.c == lo[d].c) {
        if (l.e != lo[d].e) throw std::runtime_error("axpy extent mismatch");
        sp.s1[d] = l.s;
        found = true;
      }
    if (!found) throw std::runtime_error("axpy label sets differ");
  }
  if (sp.ndim == 0) {
    sp.ndim = 1;
    sp.ext[0] = 1;
    sp.s0[0] = sp.s1[0] = 0;
  }
  launch_axpy_strided(O.base, A.base, sp, op.alpha, st_);
  stats.axpys++;
}

void Executor::run(const Prog& p) {
  // live ranges of temporaries owned by this run
  std::map<int, int> first_write, last_use;
  for (int i = 0; i < (int)p.size(); ++i) {
    const Op& op = p[i];
    if (!first_write.count(op.out.t)) first_write[op.out.t] = i;
    last_use[op.out.t] = i;
    last_use[op.a.t] = i;
    if (op.kind == 'C') last_use[op.b.t] = i;
  }
  const int64_t tc_calls_at_start = stats.tc_calls;
  // slices cached for amplitude-dependent tensors this run rewrites are stale
  frozen_run_ = false;
  for (const Op& op : p)
    if (frozen_tensors.count(op.out.t)) {
      frozen_run_ = true;
      if (ts_[op.out.t].p) drop_cache_range(ts_[op.out.t].p, numel(op.out.t));
    }
  std::set<int> run_temps;
  for (auto& kv : first_write) {
    int t = kv.first;
    const TS& s = ts_[t];
    if (!s.p) run_temps.insert(t);
  }
  // CCSD_OP_TIMING=1: time every op with events on the stream and print one line per op
  static const bool op_timing = [] {
    const char* e = getenv("CCSD_OP_TIMING");
    return e && e[0] == '1';
  }();
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (op_timing) {
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
  }
  // a run that ends by an exception leaves no temporary bound: the call's TempScope
  // releases their memory, and the next run must allocate them afresh
  struct ResetTemps {
    std::vector<TS>& ts;
    const std::set<int>& temps;
    int uncaught = std::uncaught_exceptions();
    ~ResetTemps() {
      if (std::uncaught_exceptions() > uncaught)
        for (int t : temps) ts[t].p = nullptr;
    }
  } reset_temps{ts_, run_temps};
  for (int i = 0; i < (int)p.size(); ++i) {
    const Op& op = p[i];
    if (op_timing) CK(cudaEventRecord(ev0, st_));
    double f0 = stats.gemm_flops + stats.tc_flops;
    auto check_read = [&](int t) {
      if (!ts_[t].p) throw std::runtime_error("read before write: " + g_.T[t].name);
    };
    check_read(op.a.t);
    if (op.kind == 'C') check_read(op.b.t);
    if (first_write[op.out.t] == i) {
      int t = op.out.t;
      if (run_temps.count(t)) {
        ts_[t].p = tmp_alloc(numel(t));
        ts_[t].owned = false;
        ts_[t].zstride = -1;
      }
      zero_tensor(t);
    }
    if (op.kind == 'C')
      exec_contract(op);
    else
      exec_axpy(op);
    if (op_timing) {
      CK(cudaEventRecord(ev1, st_));
      CK(cudaEventSynchronize(ev1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev0, ev1));
      double fl = stats.gemm_flops + stats.tc_flops - f0;
      fprintf(stderr, "[op %3d] %c %-14s %-8s <- %-14s %-8s %-14s %-8s %9.3f ms %10.3f GF/s\n", i, op.kind,
              g_.T[op.out.t].name.c_str(), op.lo.c_str(), g_.T[op.a.t].name.c_str(), op.la.c_str(),
              op.kind == 'C' ? g_.T[op.b.t].name.c_str() : "", op.kind == 'C' ? op.lb.c_str() : "", ms,
              ms > 0 ? fl / (ms * 1e6) : 0.0);
    }
    // release temporaries whose last use was this op
    auto release = [&](int t) {
      if (run_temps.count(t) && last_use[t] == i && ts_[t].p) {
        tmp_free(ts_[t].p);
        ts_[t].p = nullptr;
      }
    };
    release(op.out.t);
    release(op.a.t);
    if (op.kind == 'C') release(op.b.t);
  }
  if (op_timing) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  CK(cudaGetLastError());
  if (!capturing && stats.tc_calls != tc_calls_at_start) {
    int f = tc_error();
    if (f != 0) throw DeviceTimeout("a tensor-core kernel wait exceeded its budget");
  }
}

}  // namespace ccsd
