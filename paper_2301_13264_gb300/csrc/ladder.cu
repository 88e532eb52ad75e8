// Particle-particle ladder X[m][a][b] = sum_cd A[m][c][d] W[a][b][c][d] with
// W[a][b][c][d] = (ac|bd), evaluated in the symmetric/antisymmetric form.
//
// W is symmetric under the swap (a,c) <-> (b,d): W[b][a][d][c] = W[a][b][c][d].
// Split both operands under c <-> d, for a <= b and c <= d (packed pairs):
//   W+[ab][cd] = (W[a][b][c][d] + W[a][b][d][c]) / 2,  W-[ab][cd] = (W[a][b][c][d] - W[a][b][d][c]) / 2,
//   A+[m][cd]  = A[m][c][d] + A[m][d][c],               A-[m][cd]  = A[m][c][d] - A[m][d][c]   (c < d),
//   A+[m][cc]  = A[m][c][c],  A-[m][cc] = 0,  W+[ab][cc] = W[a][b][c][c],  W-[ab][cc] = 0.
// Then sum_cd A[m][c][d] W[a][b][c][d] = sum_{c<=d} A+ W+ + A- W-.  With
// Y+- = A+- (W+-)^T over the packed pairs, and because W+ is symmetric and W-
// antisymmetric under a <-> b,
//   X[m][a][b] = Y+[m][ab] + Y-[m][ab],   X[m][b][a] = Y+[m][ab] - Y-[m][ab]   (a < b),
//   X[m][a][a] = Y+[m][aa].
// The two products cost 2 M (v(v+1)/2)^2 multiply-adds instead of M v^4: about
// half of the unpacked contraction, exactly, for any A.
//
// Pair symmetry.  When the rows are (..., i, j) and A is a doubles vector of the
// library's layout, A[..][i][j][c][d] = A[..][j][i][d][c]; then A+ is symmetric
// and A- antisymmetric under i <-> j, hence so are Y+ and Y-, and only the rows
// i <= j (plus) and i < j (minus) are computed:
//   X[..][i][j][a][b] = Y+[..][ij][ab] + Y-[..][ij][ab]  and  X[..][j][i][b][a] = the same (i <= j),
//   X[..][i][j][b][a] = Y+ - Y-                          and  X[..][j][i][a][b] = the same,
// which brings the ladder to o^2 v^4 / 4 multiply-adds per vector.  Every ladder
// operand in the library's programs has this symmetry (amplitudes, trial vectors
// and the adjoints of the pair-symmetrised doubles residual); the executor uses
// the reduced rows when the operand's labels have the (.., i, j, c, d) pattern
// with i, j occupied.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <stdexcept>
#include <string>
#include <vector>

#include "alloc.h"
#include "exec.h"
#include "tcgen05.cuh"

namespace ccsd {

namespace {

__global__ void k_pair_table(int v, int2* pairs) {
  // packed index of (c, d), c <= d: p = d (d + 1) / 2 + c
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < v; d += gridDim.x * blockDim.x)
    for (int c = 0; c <= d; ++c) pairs[d * (d + 1) / 2 + c] = make_int2(c, d);
}

__device__ __forceinline__ void put(bool bf16, int S, int64_t plane, __nv_bfloat16* d16, double* d64, int64_t at,
                                    double x) {
  if (bf16) {
    unsigned short q[3];
    tc::split_bf16(x, S, q);  // integer and FP32 operations (the FP64 pipe issues 2 per clock per SM)
#pragma unroll
    for (int s = 0; s < 3; ++s)
      if (s < S) d16[s * plane + at] = __ushort_as_bfloat16(q[s]);
  } else {
    d64[at] = x;
  }
}

// A+- over rows (strided gather, ext/s1) and packed column pairs.
template <bool BF16>
__global__ void k_pack_a_pm(const double* __restrict__ A, Strided rows, int64_t sc, int64_t sd,
                            const int2* __restrict__ pairs, int np, int64_t nrows, int S, int64_t ld, int64_t plane,
                            __nv_bfloat16* p16, __nv_bfloat16* m16, double* p64, double* m64) {
  const int64_t total = nrows * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / np;
    const int p = (int)(idx - row * np);
    int64_t r = row, off = 0;
    for (int d = rows.ndim - 1; d >= 0; --d) {
      const int64_t e = rows.ext[d];
      off += (r % e) * rows.s1[d];
      r /= e;
    }
    const int2 cd = pairs[p];
    const double x = A[off + cd.x * sc + cd.y * sd];
    double pl, mi;
    if (cd.x == cd.y) {
      pl = x;
      mi = 0.0;
    } else {
      const double y = A[off + cd.y * sc + cd.x * sd];
      pl = x + y;
      mi = x - y;
    }
    put(BF16, S, plane, p16, p64, row * ld + p, pl);
    put(BF16, S, plane, m16, m64, row * ld + p, mi);
  }
}

// W+- from the contiguous W[a][b][c][d]: rows (a <= b), columns (c <= d).
template <bool BF16>
__global__ void k_pack_w_pm(const double* __restrict__ W, int64_t v, const int2* __restrict__ pairs, int np, int S,
                            int64_t ld, int64_t plane, __nv_bfloat16* p16, __nv_bfloat16* m16, double* p64,
                            double* m64) {
  const int64_t total = (int64_t)np * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / np;
    const int p = (int)(idx - row * np);
    const int2 ab = pairs[row], cd = pairs[p];
    const int64_t base = ((int64_t)ab.x * v + ab.y) * v * v;
    const double x = W[base + (int64_t)cd.x * v + cd.y];
    double pl, mi;
    if (cd.x == cd.y) {
      pl = x;
      mi = 0.0;
    } else {
      const double y = W[base + (int64_t)cd.y * v + cd.x];
      pl = 0.5 * (x + y);
      mi = 0.5 * (x - y);
    }
    put(BF16, S, plane, p16, p64, row * ld + p, pl);
    put(BF16, S, plane, m16, m64, row * ld + p, mi);
  }
}

// out[m][a][b] += alpha (Y+ + Y-), out[m][b][a] += alpha (Y+ - Y-) for a < b; a = b: alpha Y+.
__global__ void k_ladder_unpack(const double* __restrict__ Yp, const double* __restrict__ Ym, int64_t ldy,
                                Strided rows, int64_t sa, int64_t sb, const int2* __restrict__ pairs, int np,
                                int64_t nrows, double* out, double alpha) {
  const int64_t total = nrows * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / np;
    const int p = (int)(idx - row * np);
    int64_t r = row, off = 0;
    for (int d = rows.ndim - 1; d >= 0; --d) {
      const int64_t e = rows.ext[d];
      off += (r % e) * rows.s0[d];
      r /= e;
    }
    const int2 ab = pairs[p];
    const double yp = Yp[row * ldy + p], ym = Ym[row * ldy + p];
    if (ab.x == ab.y) {
      out[off + ab.x * (sa + sb)] += alpha * yp;
    } else {
      out[off + ab.x * sa + ab.y * sb] += alpha * (yp + ym);
      out[off + ab.y * sa + ab.x * sb] += alpha * (yp - ym);
    }
  }
}

// Pair-symmetric rows: row r = (prefix, i <= j) with A offset offA[r]; sign +1 packs
// A+ (A[c][d] + A[d][c], diagonal A[c][c]), sign -1 packs A- (A[c][d] - A[d][c], diagonal 0).
template <bool BF16>
__global__ void k_pack_a_sym(const double* __restrict__ A, const int64_t* __restrict__ offA, int64_t nrows,
                             int64_t sc, int64_t sd, const int2* __restrict__ pairs, int np, double sign, int S,
                             int64_t ld, int64_t plane, __nv_bfloat16* o16, double* o64) {
  const int64_t total = nrows * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / np;
    const int p = (int)(idx - row * np);
    const int2 cd = pairs[p];
    const int64_t off = offA[row];
    const double x = A[off + cd.x * sc + cd.y * sd];
    double val;
    if (cd.x == cd.y)
      val = (sign > 0) ? x : 0.0;
    else
      val = x + sign * A[off + cd.y * sc + cd.x * sd];
    put(BF16, S, plane, o16, o64, row * ld + p, val);
  }
}

// out += alpha X for the four (or fewer, on diagonals) elements each (row, ab) determines.
__global__ void k_ladder_unpack_sym(const double* __restrict__ Yp, const double* __restrict__ Ym, int64_t ldy,
                                    const int64_t* __restrict__ offIJ, const int64_t* __restrict__ offJI,
                                    const unsigned char* __restrict__ same, int64_t sa, int64_t sb,
                                    const int2* __restrict__ pairs, int np, int64_t nrows, double* out, double alpha) {
  const int64_t total = nrows * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / np;
    const int p = (int)(idx - row * np);
    const int2 ab = pairs[p];
    const double yp = Yp[row * ldy + p], ym = Ym[row * ldy + p];
    const int64_t oij = offIJ[row], oji = offJI[row];
    const int64_t ab_ = ab.x * sa + ab.y * sb, ba_ = ab.y * sa + ab.x * sb;
    if (same[row]) {  // i == j
      out[oij + ab_] += alpha * (yp + ym);
      if (ab.x != ab.y) out[oij + ba_] += alpha * (yp - ym);
    } else if (ab.x == ab.y) {  // i < j, a == b
      out[oij + ab_] += alpha * yp;
      out[oji + ab_] += alpha * yp;
    } else {
      out[oij + ab_] += alpha * (yp + ym);
      out[oji + ba_] += alpha * (yp + ym);
      out[oij + ba_] += alpha * (yp - ym);
      out[oji + ab_] += alpha * (yp - ym);
    }
  }
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace

const int2* Executor::pair_table() {
  if (!pairs_) {
    const int np = v_ * (v_ + 1) / 2;
    pairs_ = dev_alloc(np * sizeof(int2), st_, false);
    count_launches(1);
    k_pair_table<<<(v_ + 127) / 128, 128, 0, st_>>>(v_, (int2*)pairs_);
  }
  return (const int2*)pairs_;
}

bool Executor::try_ladder(const Op& op) {
  if (op.kind != 'C' || ladder_w_ < 0 || op.b.t != ladder_w_ || op.b.blk != "vvvv") return false;
  const std::string &lo = op.lo, &la = op.la, &lb = op.lb;
  if (lb.size() != 4) return false;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (lb[i] == lb[j]) return false;
  auto in = [](const std::string& s, char c) { return s.find(c) != std::string::npos; };
  // W[a][b][c][d] = (ac|bd) = W[c][d][a][b]: the output pair (n1, n2) and the
  // summed pair (k1, k2) are either (lb0, lb1 | lb2, lb3) or (lb2, lb3 | lb0, lb1)
  char n1, n2, k1, k2;
  if (in(lo, lb[0]) && in(lo, lb[1]) && !in(lo, lb[2]) && !in(lo, lb[3]) && in(la, lb[2]) && in(la, lb[3]) &&
      !in(la, lb[0]) && !in(la, lb[1])) {
    n1 = lb[0], n2 = lb[1], k1 = lb[2], k2 = lb[3];
  } else if (in(lo, lb[2]) && in(lo, lb[3]) && !in(lo, lb[0]) && !in(lo, lb[1]) && in(la, lb[0]) && in(la, lb[1]) &&
             !in(la, lb[2]) && !in(la, lb[3])) {
    n1 = lb[2], n2 = lb[3], k1 = lb[0], k2 = lb[1];
  } else {
    return false;
  }
  SView O = resolve(op.out), A = resolve(op.a);
  auto lO = merge(O, lo), lA = merge(A, la);
  if (lO.size() != lo.size() || lA.size() != la.size()) return false;  // no diagonals here
  // rows: the labels of A other than (k1, k2), in A's order; out must carry the same
  Strided rows;
  rows.ndim = 0;
  int64_t nrows = 1, sc = 0, sd = 0, sa = 0, sb = 0;
  for (auto& l : lA) {
    if (l.c == k1) {
      sc = l.s;
      continue;
    }
    if (l.c == k2) {
      sd = l.s;
      continue;
    }
    bool found = false;
    for (auto& m : lO)
      if (m.c == l.c) {
        if (m.e != l.e || rows.ndim >= kMaxDims) return false;
        rows.ext[rows.ndim] = l.e;
        rows.s1[rows.ndim] = l.s;
        rows.s0[rows.ndim] = m.s;
        rows.ndim++;
        nrows *= l.e;
        found = true;
      }
    if (!found) return false;
  }
  for (auto& m : lO) {
    if (m.c == n1) sa = m.s;
    if (m.c == n2) sb = m.s;
    if ((m.c == n1 || m.c == n2) && m.e != v_) return false;
  }
  for (auto& l : lA)
    if ((l.c == k1 || l.c == k2) && l.e != v_) return false;
  if ((int)lO.size() != rows.ndim + 2) return false;
  if (rows.ndim == 0) {
    rows.ndim = 1;
    rows.ext[0] = 1;
    rows.s0[0] = rows.s1[0] = 0;
  }
  const int np = v_ * (v_ + 1) / 2;
  // pair-symmetric pattern: A labels (prefix.., x, y, k1, k2), out labels (prefix.., x, y, n1, n2), x, y occupied
  bool sym = false;
  std::vector<int64_t> offA, offIJ, offJI;
  std::vector<unsigned char> same;
  {
    const size_t L = la.size();
    if (L >= 4 && lo.size() == L && la[L - 2] == k1 && la[L - 1] == k2 && lo[L - 2] == n1 && lo[L - 1] == n2 &&
        la.substr(0, L - 2) == lo.substr(0, L - 2) && la[L - 4] != la[L - 3] && lA[L - 4].e == o_ &&
        lA[L - 3].e == o_) {
      sym = true;
      int64_t npre = 1;
      for (size_t d = 0; d + 4 < L; ++d) npre *= lA[d].e;
      for (int64_t pre = 0; pre < npre; ++pre) {
        int64_t r = pre, oa = 0, oo = 0;
        for (int d = (int)L - 5; d >= 0; --d) {
          const int64_t c = r % lA[d].e;
          r /= lA[d].e;
          oa += c * lA[d].s;
          oo += c * lO[d].s;
        }
        for (int i = 0; i < o_; ++i)
          for (int j = i; j < o_; ++j) {
            offA.push_back(oa + i * lA[L - 4].s + j * lA[L - 3].s);
            offIJ.push_back(oo + i * lO[L - 4].s + j * lO[L - 3].s);
            offJI.push_back(oo + j * lO[L - 4].s + i * lO[L - 3].s);
            same.push_back(i == j ? 1 : 0);
          }
      }
      nrows = (int64_t)offA.size();
    }
  }
  const double flops_each = 2.0 * (double)nrows * np * np;
  const bool mixed = (prec_ == PREC_MIXED && flops_each >= tc_min_flops);
  const bool fp64tc = (prec_ == PREC_FP64_TC && flops_each >= tc_min_flops);
  const int2* pairs = pair_table();
  const double* Wp = ts_[ladder_w_].p;
  // row tables of the pair-symmetric form: device copies kept for the executor's
  // life (one per distinct table), so that a run issues no host-to-device copy
  const int64_t* dOffA = nullptr;
  const int64_t* dOffIJ = nullptr;
  const int64_t* dOffJI = nullptr;
  const unsigned char* dSame = nullptr;
  if (sym) {
    const size_t n8 = offA.size() * sizeof(int64_t);
    const LadderTables* tab = nullptr;
    for (const LadderTables& t : ladder_tables_)
      if (t.offA == offA && t.offIJ == offIJ && t.offJI == offJI && t.same == same) tab = &t;
    if (!tab) {
      LadderTables t{offA, offIJ, offJI, same, nullptr};
      t.dev = dev_alloc(3 * n8 + same.size() + 16, st_, false);
      char* base = (char*)t.dev;
      cudaMemcpy(base, offA.data(), n8, cudaMemcpyHostToDevice);
      cudaMemcpy(base + n8, offIJ.data(), n8, cudaMemcpyHostToDevice);
      cudaMemcpy(base + 2 * n8, offJI.data(), n8, cudaMemcpyHostToDevice);
      cudaMemcpy(base + 3 * n8, same.data(), same.size(), cudaMemcpyHostToDevice);
      ladder_tables_.push_back(std::move(t));
      tab = &ladder_tables_.back();
    }
    const char* base = (const char*)tab->dev;
    dOffA = (const int64_t*)base;
    dOffIJ = (const int64_t*)(base + n8);
    dOffJI = (const int64_t*)(base + 2 * n8);
    dSame = (const unsigned char*)(base + 3 * n8);
  }
  double* Yp = tmp_alloc(nrows * np);
  double* Ym = tmp_alloc(nrows * np);
  const int S = (splits_ >= 3) ? 3 : 2;
  const int64_t Kp = ((int64_t)np + 63) / 64 * 64;
  // constant W+- (built once per precision)
  WPM* w = nullptr;
  for (auto& e : wpm_)
    if (e.mixed == mixed && e.S == (mixed ? S : 0)) w = &e;
  if (!w) {
    WPM e;
    e.mixed = mixed;
    e.S = mixed ? S : 0;
    if (mixed) {
      e.rows_p = ((int64_t)np + 255) / 256 * 256;
      e.ld = Kp;
      size_t bytes = (size_t)S * e.rows_p * Kp * sizeof(__nv_bfloat16);
      e.plus = dev_alloc(bytes, st_, false);
      try {
        e.minus = dev_alloc(bytes, st_, false);
      } catch (...) {
        dev_free(e.plus, st_, false);
        throw;
      }
      cudaMemsetAsync(e.plus, 0, bytes, st_);
      cudaMemsetAsync(e.minus, 0, bytes, st_);
      count_launches(1);
      k_pack_w_pm<true><<<grid_of((int64_t)np * np), 256, 0, st_>>>(Wp, v_, pairs, np, S, Kp, e.rows_p * Kp,
                                                                  (__nv_bfloat16*)e.plus, (__nv_bfloat16*)e.minus,
                                                                  nullptr, nullptr);
      e.bytes = 2 * bytes;
    } else {
      e.rows_p = np;
      e.ld = np;
      size_t bytes = (size_t)np * np * sizeof(double);
      e.plus = dev_alloc(bytes, st_, false);
      try {
        e.minus = dev_alloc(bytes, st_, false);
      } catch (...) {
        dev_free(e.plus, st_, false);
        throw;
      }
      count_launches(1);
      k_pack_w_pm<false><<<grid_of((int64_t)np * np), 256, 0, st_>>>(Wp, v_, pairs, np, 0, np, 0, nullptr, nullptr,
                                                                   (double*)e.plus, (double*)e.minus);
      e.bytes = 2 * bytes;
    }
    cache_bytes_ += e.bytes;
    wpm_.push_back(e);
    w = &wpm_.back();
  }
  int pm_part = 0;  // 0: the + GEMM, 1: the - GEMM
  auto prof_begin = [&](ProfRec& rec) {
    if (!profiling_) return;
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, st_);
    rec.flops = flops_each;
    rec.m = nrows;
    rec.n = np;
    rec.k = np;
    rec.label = op_label(op) + (pm_part == 0 ? " (pp-ladder, + pairs)" : " (pp-ladder, - pairs)");
    pm_part ^= 1;
  };
  auto prof_end = [&](ProfRec& rec, bool tc) {
    if (!profiling_) return;
    cudaEventRecord(rec.b, st_);
    rec.tc = tc;
    rec.engine = !tc ? 0 : mixed ? 1 : 2;
    rec.ladder = true;
    rec.issued = tc ? last_tc_issued : flops_each;
    prof_.push_back(rec);
  };
  if (mixed) {
    const int64_t rows_p = (nrows + 127) / 128 * 128;
    size_t bytes = (size_t)S * rows_p * Kp * sizeof(__nv_bfloat16);
    void* ap = dev_alloc(bytes, st_, true);
    void* am = nullptr;
    try {
      am = dev_alloc(bytes, st_, true);
    } catch (...) {
      dev_free(ap, st_, true);
      throw;
    }
    cudaMemsetAsync(ap, 0, bytes, st_);
    cudaMemsetAsync(am, 0, bytes, st_);
    if (sym) {
      count_launches(2);
      k_pack_a_sym<true><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, dOffA, nrows, sc, sd, pairs, np, 1.0, S, Kp,
                                                               rows_p * Kp, (__nv_bfloat16*)ap, nullptr);
      k_pack_a_sym<true><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, dOffA, nrows, sc, sd, pairs, np, -1.0, S, Kp,
                                                               rows_p * Kp, (__nv_bfloat16*)am, nullptr);
    } else {
      count_launches(1);
      k_pack_a_pm<true><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, rows, sc, sd, pairs, np, nrows, S, Kp,
                                                              rows_p * Kp, (__nv_bfloat16*)ap, (__nv_bfloat16*)am,
                                                              nullptr, nullptr);
    }
    ProfRec r1{}, r2{};
    nvtxRangePushA("pp_ladder");  // lets a profiler select the ladder GEMMs
    prof_begin(r1);
    tc_run((__nv_bfloat16*)ap, rows_p, (__nv_bfloat16*)w->plus, w->rows_p, np, Kp, S, (int)nrows, np, Yp, np, 1,
           1.0, 0.0);
    prof_end(r1, true);
    prof_begin(r2);
    tc_run((__nv_bfloat16*)am, rows_p, (__nv_bfloat16*)w->minus, w->rows_p, np, Kp, S, (int)nrows, np, Ym, np, 1,
           1.0, 0.0);
    prof_end(r2, true);
    nvtxRangePop();
    dev_free(ap, st_, true);
    dev_free(am, st_, true);
    stats.tc_calls += 2;
    stats.tc_flops += 2 * flops_each;
  } else {
    double* ap = tmp_alloc(nrows * np);
    double* am = tmp_alloc(nrows * np);
    if (sym) {
      count_launches(2);
      k_pack_a_sym<false><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, dOffA, nrows, sc, sd, pairs, np, 1.0, 0, np,
                                                                0, nullptr, ap);
      k_pack_a_sym<false><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, dOffA, nrows, sc, sd, pairs, np, -1.0, 0, np,
                                                                0, nullptr, am);
    } else {
      count_launches(1);
      k_pack_a_pm<false><<<grid_of(nrows * np), 256, 0, st_>>>(A.base, rows, sc, sd, pairs, np, nrows, 0, np, 0,
                                                               nullptr, nullptr, ap, am);
    }
    for (int pm = 0; pm < 2; ++pm) {
      GemmArgs g;
      g.batch = 1;
      g.M = (int)nrows;
      g.N = np;
      g.K = np;
      g.A = pm == 0 ? ap : am;
      g.sAb = 0;
      g.sAm = np;
      g.sAk = 1;
      g.B = (const double*)(pm == 0 ? w->plus : w->minus);
      g.sBb = 0;
      g.sBn = np;
      g.sBk = 1;
      g.C = pm == 0 ? Yp : Ym;
      g.sCb = 0;
      g.sCm = np;
      g.sCn = 1;
      g.alpha = 1.0;
      g.beta = 0.0;
      ProfRec r{};
      prof_begin(r);
      if (fp64tc) {
        // FP64-grade tensor-core products; the fixed-point slices of W+- stay cached
        Strided ga, gw;
        ga.ndim = gw.ndim = 2;
        ga.ext[0] = nrows;
        gw.ext[0] = np;
        ga.ext[1] = gw.ext[1] = np;
        ga.s1[0] = gw.s1[0] = np;
        ga.s1[1] = gw.s1[1] = 1;
        ga.s0[0] = ga.s0[1] = gw.s0[0] = gw.s0[1] = 0;
        if (!fp64tc_contract((int)nrows, np, np, g.A, ga, g.B, gw, g.C, np, 1, 1.0, 0.0, false, true))
          launch_dgemm(g, st_);
      } else {
        launch_dgemm(g, st_);
      }
      prof_end(r, fp64tc);
    }
    tmp_free(ap);
    tmp_free(am);
    if (fp64tc) {
      stats.tc_calls += 2;
      stats.tc_flops += 2 * flops_each;
    } else {
      stats.gemm_calls += 2;
      stats.gemm_flops += 2 * flops_each;
    }
  }
  count_launches(1);
  if (sym)
    k_ladder_unpack_sym<<<grid_of(nrows * np), 256, 0, st_>>>(Yp, Ym, np, dOffIJ, dOffJI, dSame, sa, sb, pairs, np,
                                                              nrows, O.base, op.alpha);
  else
    k_ladder_unpack<<<grid_of(nrows * np), 256, 0, st_>>>(Yp, Ym, np, rows, sa, sb, pairs, np, nrows, O.base,
                                                          op.alpha);
  tmp_free(Yp);
  tmp_free(Ym);
  stats.ladders++;
  return true;
}

}  // namespace ccsd
