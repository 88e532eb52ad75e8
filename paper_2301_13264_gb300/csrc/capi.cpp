// C ABI: handle, solvers (ground state, Lambda, EOM, coupling multipliers),
// coupling densities and derivative couplings.  All vector arithmetic runs in
// the library's CUDA kernels; the host only solves the small subspace problems.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ccsd.h"
#include "alloc.h"
#include "exec.h"
#include "kernels.cuh"
#include "mlp.h"
#include "orbital.h"
#include "programs.h"
#include "small_linalg.h"
#include "subspace.h"

static_assert(ccsd::mlp::kParams == CCSD_MLP_PARAMS, "model size");

using namespace ccsd;

namespace {

struct Err : std::runtime_error {
  ccsd_status code;
  Err(ccsd_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// message of the last failed call made without a handle (per thread)
thread_local std::string g_last_error;

#define CUDA_OK(x)                                                                                 \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ == cudaErrorMemoryAllocation) throw Err(CCSD_ERR_OOM, std::string(#x ": out of memory")); \
    if (e_ != cudaSuccess) throw Err(CCSD_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DevBuf {
  double* p = nullptr;
  int64_t n = 0;
  DevBuf() = default;
  explicit DevBuf(int64_t n_) { alloc(n_); }
  // device memory of the handle whose call is running (its allocator callbacks, else
  // cudaMalloc); released on the handle's stream in the callbacks' case
  void alloc(int64_t n_) {
    release();
    p = (double*)dev_alloc(std::max<int64_t>(n_, 1) * sizeof(double), active_stream(), false);
    n = n_;
  }
  void release() {
    dev_free(p, active_stream(), false);
    p = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

}  // namespace

struct ccsd_ctx {
  ccsd_options opt;
  int o = 0, v = 0, naux = 0, n = 0;
  VecShape vs;
  int64_t dim = 0, n1 = 0;
  cudaStream_t st = 0;
  int device = 0;  // the GPU that was current at ccsd_create: all of the handle's memory lives there
  DeviceAllocator allocator;  // the caller's allocator callbacks (none: the CUDA runtime)
  Programs P;
  std::unique_ptr<Executor> ex;
  DevBuf eps, h, B, ones;
  DevBuf t, lam, eta, omega_buf, escal, seedE, gsc;  // amplitudes, multipliers, scratch
  std::vector<std::unique_ptr<DevBuf>> R, L;
  std::vector<double> r0, omega;
  bool have_ground = false, have_right = false, have_left = false;
  bool cache_at_t = false;  // primal intermediates correspond to the converged t
  double e_ccsd = 0.0;
  std::string err;
  // densities of the last pair
  int dens_k = -1, dens_l = -1;
  DevBuf Dd, Zd;
  // device staging of host-memory trial vectors for ccsd_jacobian_transform, kept between calls
  // (grown as needed) so that a host-pointer call allocates and frees nothing in steady state
  DevBuf stage_x, stage_y;
  long long prof_launch0 = 0;
  DevBuf guess_model;  // MLP model (floats) for the starting doubles, or empty
  DevBuf mult_model;   // MLP model for the starting doubles of the multiplier solves, or empty
  int iters_ground = 0, iters_lambda = 0, iters_zeta = 0;  // of the last solves
  // orbital relaxation (relax_orbitals): Hartree-Fock programs on the handle's (h, B)
  std::unique_ptr<HFPrograms> hfp;
  std::unique_ptr<Executor> hx;
  std::vector<double> kbar;  // kappa-bar of the last pair [o][v]
};

namespace {

void sync(ccsd_ctx* c) { CUDA_OK(cudaStreamSynchronize(c->st)); }

// G[p][q] = <X_p|Y_q> on the host
std::vector<double> gram(ccsd_ctx* c, const double* X, int64_t ldx, int np, const double* Y, int64_t ldy, int nq) {
  DevBuf G(np * nq);
  double* work = c->ex->scratch(wdot_work_size(np, nq));
  launch_wdot(c->vs, X, ldx, np, Y, ldy, nq, G.p, nq, work, c->st);
  std::vector<double> h(np * nq);
  CUDA_OK(cudaMemcpyAsync(h.data(), G.p, np * nq * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  return h;
}

double maxabs(ccsd_ctx* c, const double* x, int64_t n) {
  DevBuf out(2);
  launch_maxabs(n, x, out.p, c->ex->scratch(1024), c->st);
  double r;
  CUDA_OK(cudaMemcpyAsync(&r, out.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  return r;
}

// Y[q] = sum_p coef[p][q] X[p] (coef on host, row-major np x nq)
void lincomb(ccsd_ctx* c, const double* X, int64_t ldx, int np, const std::vector<double>& coef, double* Y,
             int64_t ldy, int nq, bool acc) {
  DevBuf cd(np * nq);
  CUDA_OK(cudaMemcpyAsync(cd.p, coef.data(), np * nq * sizeof(double), cudaMemcpyHostToDevice, c->st));
  launch_lincomb(c->vs, X, ldx, np, cd.p, nq, Y, ldy, nq, acc, c->st);
  sync(c);  // coefficient buffer is released on return
}

// ---------------------------------------------------------------------------
// program drivers
// ---------------------------------------------------------------------------

// Omega(t) -> om, energy (host).  Updates the cached primal intermediates.
double forward(ccsd_ctx* c, const double* t, double* om) {
  auto& cp = c->P.cp;
  Executor& ex = *c->ex;
  ex.invalidate_frozen();  // new amplitudes: slices of the old ones and their intermediates are stale
  ex.set_nvec(1);
  ex.bind(cp.t1, const_cast<double*>(t));
  ex.bind(cp.t2, const_cast<double*>(t) + c->n1);
  ex.bind(cp.O1, om);
  ex.bind(cp.O2, om + c->n1);
  ex.bind(cp.E, c->escal.p);
  ex.run(cp.fwd_t);
  double e;
  CUDA_OK(cudaMemcpyAsync(&e, c->escal.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  c->cache_at_t = (t == c->t.p);
  return e;
}

void ensure_cache(ccsd_ctx* c) {
  if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
  if (!c->cache_at_t) {
    DevBuf om(c->dim);
    forward(c, c->t.p, om.p);
  }
  auto& cp = c->P.cp;
  c->ex->bind(cp.t1, c->t.p);
  c->ex->bind(cp.t2, c->t.p + c->n1);
}

// Y = A X for nvec vectors ([nvec][dim])
void right_block(ccsd_ctx* c, const double* X, double* Y, int nvec) {
  ensure_cache(c);
  Executor& ex = *c->ex;
  auto& P = c->P;
  ex.set_nvec(nvec);
  ex.bind(P.zR1, const_cast<double*>(X), c->dim);
  ex.bind(P.zR2, const_cast<double*>(X) + c->n1, c->dim);
  ex.bind(P.zAR1, Y, c->dim);
  ex.bind(P.zAR2, Y + c->n1, c->dim);
  ex.bind(P.zAE, c->gsc.p);
  ex.run(P.jvp_z);
}

// Y = (X^T A)^T for nvec vectors; with eseed != 0 adds eseed * eta (used for eta itself)
// the left transform with caller-provided work arrays W, G ([nvec][dim] each) and
// a zero energy seed: no allocation, no host copy, no synchronisation
void left_block_into(ccsd_ctx* c, const double* X, double* Y, int nvec, double* W, double* G) {
  Executor& ex = *c->ex;
  auto& P = c->P;
  ex.set_nvec(nvec);
  launch_weight(c->vs, X, W, nvec, c->dim, c->st);
  CUDA_OK(cudaMemsetAsync(c->seedE.p, 0, nvec * sizeof(double), c->st));
  ex.bind(P.zL1, W, c->dim);
  ex.bind(P.zL2, W + c->n1, c->dim);
  ex.bind(P.zLE, c->seedE.p);
  ex.bind(P.zLA1, G, c->dim);
  ex.bind(P.zLA2, G + c->n1, c->dim);
  ex.run(P.vjp_z);
  launch_packed_grad(c->vs, G, Y, nvec, c->dim, c->st);
}

void left_block(ccsd_ctx* c, const double* X, double* Y, int nvec, double eseed = 0.0) {
  ensure_cache(c);
  Executor& ex = *c->ex;
  auto& P = c->P;
  ex.set_nvec(nvec);
  DevBuf W(nvec * c->dim), G(nvec * c->dim);
  launch_weight(c->vs, X, W.p, nvec, c->dim, c->st);
  std::vector<double> es(nvec, eseed);
  CUDA_OK(cudaMemcpyAsync(c->seedE.p, es.data(), nvec * sizeof(double), cudaMemcpyHostToDevice, c->st));
  ex.bind(P.zL1, W.p, c->dim);
  ex.bind(P.zL2, W.p + c->n1, c->dim);
  ex.bind(P.zLE, c->seedE.p);
  ex.bind(P.zLA1, G.p, c->dim);
  ex.bind(P.zLA2, G.p + c->n1, c->dim);
  ex.run(P.vjp_z);
  launch_packed_grad(c->vs, G.p, Y, nvec, c->dim, c->st);
  sync(c);
}

// y = sum_nu d^2(g0 E + <g|Omega>)/dt dt_nu r_nu (packed)
void hess_right(ccsd_ctx* c, double g0, const double* g, const double* r, double* y) {
  ensure_cache(c);
  Executor& ex = *c->ex;
  auto& P = c->P;
  ex.set_nvec(1);
  DevBuf W(c->dim), G(c->dim), s0(1);
  launch_weight(c->vs, g, W.p, 1, c->dim, c->st);
  CUDA_OK(cudaMemcpyAsync(s0.p, &g0, sizeof(double), cudaMemcpyHostToDevice, c->st));
  ex.bind(P.hG1, W.p);
  ex.bind(P.hG2, W.p + c->n1);
  ex.bind(P.hG0, s0.p);
  ex.bind(P.hR1, const_cast<double*>(r));
  ex.bind(P.hR2, const_cast<double*>(r) + c->n1);
  ex.bind(P.hF1, G.p);
  ex.bind(P.hF2, G.p + c->n1);
  ex.run(P.hvp);
  launch_packed_grad(c->vs, G.p, y, 1, c->dim, c->st);
  sync(c);
}

// ---------------------------------------------------------------------------
// DIIS
// ---------------------------------------------------------------------------
struct Diis {
  ccsd_ctx* c;
  int cap;
  DevBuf X, E;             // [cap][dim] ring buffers of vectors and errors
  std::vector<double> Bm;  // cap x cap Gram matrix of stored errors
  int m = 0, next = 0;
  Diis(ccsd_ctx* c_, int cap_) : c(c_), cap(std::max(cap_, 1)), Bm(cap * cap, 0.0) {
    X.alloc(cap * c->dim);
    E.alloc(cap * c->dim);
  }
  // store (x, e) and write the extrapolated vector to out
  void step(const double* x, const double* e, double* out) {
    int slot = next;
    next = (next + 1) % cap;
    m = std::min(m + 1, cap);
    const int64_t dim = c->dim;
    CUDA_OK(cudaMemcpyAsync(X.p + slot * dim, x, dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    CUDA_OK(cudaMemcpyAsync(E.p + slot * dim, e, dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    std::vector<double> d = gram(c, E.p, dim, m, E.p + slot * dim, dim, 1);
    for (int q = 0; q < m; ++q) Bm[q * cap + slot] = Bm[slot * cap + q] = d[q];
    if (m < 2) {
      CUDA_OK(cudaMemcpyAsync(out, x, c->dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      return;
    }
    int k = m + 1;
    std::vector<double> A(k * k, 0.0), b(k, 0.0);
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(Bm[i * cap + i]));
    if (scale == 0.0) scale = 1.0;
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) A[i * k + j] = Bm[i * cap + j] / scale;
      A[i * k + m] = A[m * k + i] = -1.0;
    }
    b[m] = -1.0;
    if (!lu_solve(k, A, b)) {
      CUDA_OK(cudaMemcpyAsync(out, x, c->dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      return;
    }
    // slots 0..m-1 hold the stored vectors (ring buffer, all valid once m == cap)
    std::vector<double> coef(b.begin(), b.begin() + m);
    lincomb(c, X.p, dim, m, coef, out, dim, 1, false);
  }
};

// Sets the executor's precision for a scope.
struct PrecScope {
  ccsd_ctx* c;
  int old;
  PrecScope(ccsd_ctx* c_, int p) : c(c_), old(c_->ex->precision()) { c->ex->set_precision(p, c->opt.splits); }
  ~PrecScope() { c->ex->set_precision(old, c->opt.splits); }
};

bool refining(ccsd_ctx* c) { return c->opt.precision == CCSD_PREC_MIXED && c->opt.refine; }

// precision of the FP64 evaluations inside a mixed-precision handle (refinement residuals,
// Hamiltonian-only intermediates, densities): DFMA, or the FP64-grade tensor-core products
int fp64_prec(ccsd_ctx* c) {
  if (c->opt.precision == CCSD_PREC_FP64_TC) return PREC_FP64_TC;
  return (c->opt.precision == CCSD_PREC_MIXED && c->opt.fp64_tc) ? PREC_FP64_TC : PREC_FP64;
}

// Solve A x = -rhs by preconditioned Jacobi + DIIS (right transforms); x holds the guess on entry
int solve_right_linear(ccsd_ctx* c, const double* rhs, double* x, double tol, int maxit) {
  DevBuf res(c->dim), xn(c->dim);
  Diis diis(c, c->opt.diis_dim);
  for (int it = 1; it <= maxit; ++it) {
    right_block(c, x, res.p, 1);
    launch_axpby(c->dim, 1.0, rhs, 1.0, res.p, c->st);
    double err = maxabs(c, res.p, c->dim);
    if (!std::isfinite(err)) throw Err(CCSD_ERR_NOT_CONVERGED, "linear equations diverged");
    if (err < tol) return it;
    launch_precond(c->vs, c->eps.p, res.p, xn.p, 0.0, c->st);
    launch_axpby(c->dim, 1.0, x, -1.0, xn.p, c->st);
    diis.step(xn.p, res.p, x);
  }
  return maxit;
}

int solve_left_linear(ccsd_ctx* c, const double* rhs, double* x, double tol, bool stall_ok = false);

// x^T A = -rhs^T to the FP64 tolerance: in mixed mode with refinement the
// equations are first solved in mixed precision to tol_switch, then corrected:
// rho = rhs + A_64^T x (FP64 left transform), A^T d = -rho solved in mixed
// precision to a fraction of |rho|, x += d, until max |rho| < tol.
int solve_left_refined(ccsd_ctx* c, const double* rhs, double* x, double tol) {
  if (!refining(c)) return solve_left_linear(c, rhs, x, tol);
  int it = solve_left_linear(c, rhs, x, std::max(tol, c->opt.tol_switch), true);
  DevBuf rho(c->dim), d(c->dim);
  for (int outer = 0; outer < 20; ++outer) {
    {
      PrecScope fp64(c, fp64_prec(c));
      left_block(c, x, rho.p, 1);
    }
    launch_axpby(c->dim, 1.0, rhs, 1.0, rho.p, c->st);
    ++it;
    double err = maxabs(c, rho.p, c->dim);
    if (!std::isfinite(err)) throw Err(CCSD_ERR_NOT_CONVERGED, "refinement diverged");
    if (err < tol) return it;
    launch_precond(c->vs, c->eps.p, rho.p, d.p, 0.0, c->st);
    launch_axpby(c->dim, 0.0, d.p, -1.0, d.p, c->st);
    it += solve_left_linear(c, rho.p, d.p, std::max(1e-3 * err, 0.1 * tol), true);
    launch_axpby(c->dim, 1.0, d.p, 1.0, x, c->st);
  }
  throw Err(CCSD_ERR_NOT_CONVERGED, "FP64 refinement of the linear equations did not converge");
}

// Solve x^T A = -rhs^T by preconditioned Jacobi + DIIS; x holds the guess on entry.
// With stall_ok (the mixed phase before an FP64 refinement) the iteration also stops
// once it no longer halves the residual in 8 iterations within 100 tol: the
// mixed-precision floor, from where the refinement continues.
int solve_left_linear(ccsd_ctx* c, const double* rhs, double* x, double tol, bool stall_ok) {
  DevBuf res(c->dim), xn(c->dim);
  Diis diis(c, c->opt.diis_dim);
  double best = 1e300;
  int since_best = 0;
  for (int it = 1; it <= c->opt.max_iter; ++it) {
    left_block(c, x, res.p, 1);
    launch_axpby(c->dim, 1.0, rhs, 1.0, res.p, c->st);
    double err = maxabs(c, res.p, c->dim);
    if (!std::isfinite(err)) throw Err(CCSD_ERR_NOT_CONVERGED, "linear equations diverged");
    if (err < tol) return it;
    if (err < 0.5 * best) {
      best = err;
      since_best = 0;
    } else if (stall_ok && ++since_best >= 8 && err < 100.0 * tol) {
      return it;
    }
    launch_precond(c->vs, c->eps.p, res.p, xn.p, 0.0, c->st);
    launch_axpby(c->dim, 1.0, x, -1.0, xn.p, c->st);  // xn = x - res/D
    diis.step(xn.p, res.p, x);
  }
  throw Err(CCSD_ERR_NOT_CONVERGED, "left linear equations not converged");
}

// ---------------------------------------------------------------------------
// Davidson for the lowest nroots of A (side 0) or A^T (side 1), as a state
// machine: the caller transforms the pending trial vectors V[first, first+count)
// into AV[first, first+count) (one system at a time, or many systems in one
// batched launch) and then calls advance(), which extends the projected matrix,
// solves the subspace problem and either converges or queues new trial vectors.
// ---------------------------------------------------------------------------
class Davidson {
 public:
  Davidson(ccsd_ctx* c, int side, int nroots, double tol, const std::vector<std::unique_ptr<DevBuf>>* init)
      : side(side),
        c_(c),
        nroots_(nroots),
        tol_(tol),
        dim_(c->dim),
        maxsub_(std::max(c->opt.davidson_max_sub, 3 * nroots)),
        V(maxsub_ * c->dim),
        AV(maxsub_ * c->dim),
        X(nroots * c->dim),
        AX(nroots * c->dim),
        Rz(nroots * c->dim),
        Gd(maxsub_ * maxsub_),
        Sout(2 * nroots + maxsub_ * nroots + 1),
        Swork((subspace_work_bytes(maxsub_) + 7) / 8),
        Tg(nroots) {
    CUDA_OK(cudaMemsetAsync(Gd.p, 0, (size_t)maxsub_ * maxsub_ * sizeof(double), c->st));
    const int64_t dim = dim_;
    // guesses: the given vectors, else singles unit vectors of the lowest orbital-energy differences
    if (init && (int)init->size() >= nroots) {
      for (int g = 0; g < nroots; ++g)
        CUDA_OK(cudaMemcpyAsync(V.p + g * dim, (*init)[g]->p, dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      count = orthonormalize(nroots);
    } else {
      std::vector<double> eps(c->n);
      CUDA_OK(cudaMemcpyAsync(eps.data(), c->eps.p, c->n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      sync(c);
      std::vector<std::pair<double, int>> d1;
      for (int i = 0; i < c->o; ++i)
        for (int a = 0; a < c->v; ++a) d1.push_back({eps[c->o + a] - eps[i], i * c->v + a});
      std::stable_sort(d1.begin(), d1.end(), [](auto& x, auto& y) { return x.first < y.first; });
      // a few more start vectors than roots, so that a low root is not missed
      int ng = std::min<int>(nroots + std::min(nroots, 4), (int)d1.size());
      CUDA_OK(cudaMemsetAsync(V.p, 0, ng * dim * sizeof(double), c->st));
      std::vector<double> one(ng, 1.0);
      for (int g = 0; g < ng; ++g)
        CUDA_OK(cudaMemcpyAsync(V.p + g * dim + d1[g].second, &one[g], sizeof(double), cudaMemcpyHostToDevice,
                                c->st));
      sync(c);
      count = orthonormalize(ng);
    }
    if (count == 0) throw Err(CCSD_ERR_NOT_CONVERGED, "no Davidson start vectors");
  }

  // pending trial vectors and their transforms
  int first = 0, count = 0;
  double* vin(int q) { return V.p + (first + q) * dim_; }
  double* vout(int q) { return AV.p + (first + q) * dim_; }
  int iterations = 0;
  std::vector<double> omega;
  const int side;
  // when set (nroots values), follow the Ritz values nearest these instead of the lowest
  std::vector<double> targets;

  // transforms of the pending vectors are in place: returns true once converged
  bool advance() {
    ccsd_ctx* c = c_;
    const int64_t dim = dim_;
    ++iterations;
    // extend the projected matrix G[i][j] = <V_i|A V_j> (on the device) with the pending block
    {
      double* work = c->ex->scratch(wdot_work_size(first + count, std::max(count, first)));
      launch_wdot(c->vs, V.p, dim, first + count, AV.p + first * dim, dim, count, Gd.p + first, maxsub_, work, c->st);
      if (first > 0)
        launch_wdot(c->vs, V.p + first * dim, dim, count, AV.p, dim, first, Gd.p + (int64_t)first * maxsub_, maxsub_,
                    work, c->st);
    }
    m_ = first + count;
    count = 0;
    const int m = m_, nroots = nroots_;
    if (m < nroots) throw Err(CCSD_ERR_NOT_CONVERGED, "subspace too small");
    // the subspace eigenproblem in FP64 on the GPU: Ritz values (the lowest, or the ones nearest
    // the targets) and their coefficient vectors U[m][nroots] (subspace.cu).  A complex pair
    // a +- ib among the wanted values is usually transient (a small subspace of a non-symmetric
    // matrix); the pair's real 2-D invariant subspace is then spanned by u (inverse iteration
    // at a) and (G - a)u, which serve as the two Ritz-like vectors with shift a.  A pair that
    // survives many expansions is reported.
    const bool tgt = (int)targets.size() == nroots;
    if (tgt)
      CUDA_OK(cudaMemcpyAsync(Tg.p, targets.data(), nroots * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_subspace_step(m, Gd.p, maxsub_, nroots, tgt ? Tg.p : nullptr, Sout.p, Swork.p, c->st);
    std::vector<double> head(2 * nroots);
    double scale = 0.0;
    CUDA_OK(cudaMemcpyAsync(head.data(), Sout.p, 2 * nroots * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaMemcpyAsync(&scale, Sout.p + 2 * nroots + (int64_t)m * nroots, sizeof(double), cudaMemcpyDeviceToHost,
                            c->st));
    sync(c);
    bool cplx = false;
    omega.assign(nroots, 0.0);
    for (int k = 0; k < nroots; ++k) {
      omega[k] = head[k];
      cplx |= std::fabs(head[nroots + k]) > 1e-9 * std::max(scale, 1.0);
    }
    complex_run_ = cplx ? complex_run_ + 1 : 0;
    if (complex_run_ > 12) throw Err(CCSD_ERR_COMPLEX_ROOT, "complex eigenvalue among the wanted roots");
    const double* U = Sout.p + 2 * nroots;
    // Ritz vectors in double-float arithmetic (FP64-grade, off the FP64 pipe)
    launch_lincomb(c->vs, V.p, dim, m, U, nroots, X.p, dim, nroots, false, c->st, true);
    launch_lincomb(c->vs, AV.p, dim, m, U, nroots, AX.p, dim, nroots, false, c->st, true);
    // residuals r_k = A x_k - omega_k x_k (x_k has unit norm up to roundoff)
    std::vector<double> xn = gram(c, X.p, dim, nroots, X.p, dim, nroots);
    std::vector<int> todo;
    for (int k = 0; k < nroots; ++k) {
      double s = 1.0 / std::sqrt(xn[k * nroots + k]);
      launch_axpby(dim, s, X.p + k * dim, 0.0, X.p + k * dim, c->st);
      launch_axpby(dim, s, AX.p + k * dim, 0.0, AX.p + k * dim, c->st);
      launch_axpby(dim, 1.0, AX.p + k * dim, 0.0, Rz.p + k * dim, c->st);
      launch_axpby(dim, -omega[k], X.p + k * dim, 1.0, Rz.p + k * dim, c->st);
    }
    std::vector<double> rn = gram(c, Rz.p, dim, nroots, Rz.p, dim, nroots);
    for (int k = 0; k < nroots; ++k)
      if (std::sqrt(std::max(rn[k * nroots + k], 0.0)) > tol_) todo.push_back(k);
    if (todo.empty() && !cplx) return true;
    if (iterations >= c->opt.max_iter) throw Err(CCSD_ERR_NOT_CONVERGED, "Davidson not converged");
    int base = m_;
    if (m_ + (int)todo.size() > maxsub_) {  // restart from the current Ritz vectors
      CUDA_OK(cudaMemcpyAsync(V.p, X.p, nroots * dim * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      CUDA_OK(cudaMemsetAsync(Gd.p, 0, (size_t)maxsub_ * maxsub_ * sizeof(double), c->st));
      base = 0;
      m_ = 0;
      for (size_t q = 0; q < todo.size(); ++q)
        launch_precond(c->vs, c->eps.p, Rz.p + todo[q] * dim, V.p + (nroots + q) * dim, omega[todo[q]], c->st);
      first = 0;
      count = orthonormalize(nroots + (int)todo.size());
    } else {
      for (size_t q = 0; q < todo.size(); ++q)
        launch_precond(c->vs, c->eps.p, Rz.p + todo[q] * dim, V.p + (base + q) * dim, omega[todo[q]], c->st);
      first = base;
      count = orthonormalize((int)todo.size());
    }
    if (count == 0) throw Err(CCSD_ERR_NOT_CONVERGED, "Davidson stagnated");
    return false;
  }

  // the converged Ritz vectors (after advance() returned true)
  void results(std::vector<std::unique_ptr<DevBuf>>& out) {
    out.clear();
    for (int k = 0; k < nroots_; ++k) {
      out.emplace_back(new DevBuf(dim_));
      CUDA_OK(cudaMemcpyAsync(out[k]->p, X.p + k * dim_, dim_ * sizeof(double), cudaMemcpyDeviceToDevice, c_->st));
    }
    sync(c_);
  }

 private:
  // orthonormalise candidates in slots m_..m_+cnt-1 against V[0, m_) and each
  // other, compacting the kept ones to the front; returns the number kept
  int orthonormalize(int cnt) {
    ccsd_ctx* c = c_;
    const int64_t dim = dim_;
    int kept = 0;
    for (int q = 0; q < cnt; ++q) {
      double* x = V.p + (m_ + q) * dim;
      std::vector<double> nrm0 = gram(c, x, dim, 1, x, dim, 1);
      if (!(nrm0[0] > 0.0)) continue;
      launch_axpby(dim, 1.0 / std::sqrt(nrm0[0]), x, 0.0, x, c->st);
      int have = m_ + kept;
      for (int pass = 0; pass < 2; ++pass) {
        if (have == 0) break;
        std::vector<double> d = gram(c, V.p, dim, have, x, dim, 1);
        std::vector<double> coef(have);
        for (int i = 0; i < have; ++i) coef[i] = -d[i];
        lincomb(c, V.p, dim, have, coef, x, dim, 1, true);
      }
      std::vector<double> nrm = gram(c, x, dim, 1, x, dim, 1);
      if (nrm[0] < 1e-16) continue;
      double* dst = V.p + (m_ + kept) * dim;
      launch_axpby(dim, 1.0 / std::sqrt(nrm[0]), x, 0.0, dst, c->st);
      ++kept;
    }
    return kept;
  }

  ccsd_ctx* c_;
  int nroots_;
  double tol_;
  int64_t dim_;
  int maxsub_;
  DevBuf V, AV, X, AX, Rz;
  DevBuf Gd;     // G[i][j] = <V_i | A V_j>, maxsub x maxsub (device)
  DevBuf Sout;   // subspace step output: Ritz values, imaginary parts, U[m][nroots], scale
  DevBuf Swork;  // subspace step scratch
  DevBuf Tg;     // targets (device copy)
  int m_ = 0;
  int complex_run_ = 0;
};

// transforms of the pending Davidson vectors on the system's own stream
void transform_pending(Davidson& d, ccsd_ctx* c) {
  const int block = std::max(1, std::min(c->opt.davidson_block, 16));
  for (int s = 0; s < d.count; s += block) {
    const int nb = std::min(block, d.count - s);
    if (d.side == 0)
      right_block(c, d.vin(s), d.vout(s), nb);
    else
      left_block(c, d.vin(s), d.vout(s), nb);
  }
}

int davidson(ccsd_ctx* c, int side, int nroots, std::vector<double>& omega, std::vector<std::unique_ptr<DevBuf>>& out,
             double tol, const std::vector<std::unique_ptr<DevBuf>>* init = nullptr,
             const std::vector<double>* targets = nullptr) {
  Davidson d(c, side, nroots, tol, init);
  if (targets) d.targets = *targets;
  for (;;) {
    transform_pending(d, c);
    if (d.advance()) break;
  }
  omega = d.omega;
  d.results(out);
  return d.iterations;
}

int refine_eigenpair(ccsd_ctx* c, int side, double* x, double& w, double tol);

// CCSD_VERBOSE=1: solver progress on stderr
bool verbose_solvers() {
  static const bool v = [] {
    const char* e = getenv("CCSD_VERBOSE");
    return e && e[0] == '1';
  }();
  return v;
}

// FP64 refinement of mixed-precision eigenpairs (w, vecs) to tol_eom: defect
// correction root by root, falling back to an FP64 Davidson continuation that
// follows the same roots if a correction stalls.  Returns the transforms used.
int refine_roots(ccsd_ctx* c, int side, std::vector<double>& w, std::vector<std::unique_ptr<DevBuf>>& vecs) {
  const int nroots = (int)w.size();
  int n = 0;
  try {
    for (int k = 0; k < nroots; ++k) n += refine_eigenpair(c, side, vecs[k]->p, w[k], c->opt.tol_eom);
    return n;
  } catch (const Err& e) {
    if (e.code != CCSD_ERR_NOT_CONVERGED) throw;
  }
  PrecScope fp64(c, fp64_prec(c));
  const std::vector<double> wm = w;
  std::vector<std::unique_ptr<DevBuf>> fin;
  n += davidson(c, side, nroots, w, fin, c->opt.tol_eom, &vecs, &wm);
  vecs.swap(fin);
  return n;
}

// Davidson to tol_eom; in mixed mode with refinement the mixed-precision solution
// (to 10 tol_switch) seeds an FP64 continuation that follows the same roots.
int davidson_refined(ccsd_ctx* c, int side, int nroots, std::vector<double>& w,
                     std::vector<std::unique_ptr<DevBuf>>& out,
                     const std::vector<std::unique_ptr<DevBuf>>* init = nullptr,
                     const std::vector<double>* targets = nullptr) {
  if (!refining(c)) return davidson(c, side, nroots, w, out, c->opt.tol_eom, init, targets);
  static const bool verbose = [] {
    const char* e = getenv("CCSD_VERBOSE");
    return e && e[0] == '1';
  }();
  auto t0 = std::chrono::steady_clock::now();
  std::vector<std::unique_ptr<DevBuf>> mixed;
  const int it1 = davidson(c, side, nroots, w, mixed, std::max(c->opt.tol_eom, 10.0 * c->opt.tol_switch), init,
                           targets);
  auto t1 = std::chrono::steady_clock::now();
  const int it2 = refine_roots(c, side, w, mixed);
  out.swap(mixed);
  if (verbose) {
    auto t2 = std::chrono::steady_clock::now();
    fprintf(stderr, "[davidson side %d] mixed phase %d iterations %.2f s, FP64 refinement %d transforms %.2f s\n",
            side, it1, std::chrono::duration<double>(t1 - t0).count(), it2,
            std::chrono::duration<double>(t2 - t1).count());
  }
  return it1 + it2;
}

// Defect correction of one eigenpair (x, w) of A (side 0) or A^T (side 1) to the FP64
// residual tolerance: per outer step one FP64 transform gives r = A x - w x (w the
// Rayleigh quotient of the unit vector x); the correction d (d perpendicular to x)
// solves the projected equation P (A - w) P d = -r, P = 1 - x x^T (the Jacobi-Davidson
// correction equation), by right-preconditioned restarted GMRES with transforms at the
// handle's (mixed) precision and the preconditioner (D - w)^-1, to 1e-4 of |r|; x += d.
// For a root above the lowest, (A - w) is indefinite on the complement of x (the lower
// roots give negative eigenvalues), which GMRES handles; each outer step gains the
// mixed operator's accuracy, so two or three FP64 transforms per root replace an FP64
// Davidson continuation.  Returns the transforms used; throws if an outer step gains less than 10x.
int refine_eigenpair(ccsd_ctx* c, int side, double* x, double& w, double tol) {
  const int64_t dim = c->dim;
  constexpr int KR = 16;  // Krylov vectors per restart
  DevBuf ax(dim), r(dim), z(dim), u(dim), V((KR + 1) * dim);
  auto transform = [&](const double* in, double* out) {
    if (side == 0)
      right_block(c, in, out, 1);
    else
      left_block(c, in, out, 1);
  };
  auto project = [&](double* v) {  // v -= x <x|v>
    const double s = gram(c, x, dim, 1, v, dim, 1)[0];
    launch_axpby(dim, -s, x, 1.0, v, c->st);
  };
  auto norm = [&](const double* v) { return std::sqrt(std::max(gram(c, v, dim, 1, v, dim, 1)[0], 0.0)); };
  int n = 0;
  double last = 1e300;
  for (int outer = 0; outer < 8; ++outer) {
    const double nx = norm(x);
    launch_axpby(dim, 1.0 / nx, x, 0.0, x, c->st);
    {
      PrecScope fp64(c, fp64_prec(c));
      transform(x, ax.p);
    }
    ++n;
    w = gram(c, x, dim, 1, ax.p, dim, 1)[0];
    launch_axpby(dim, 1.0, ax.p, 0.0, r.p, c->st);
    launch_axpby(dim, -w, x, 1.0, r.p, c->st);
    const double rn = norm(r.p);
    if (verbose_solvers())
      fprintf(stderr, "[refine side %d] outer %d: w = %.12f, |r| = %.3e (%d transforms so far)\n", side, outer, w, rn, n);
    if (rn < tol) return n;
    // an outer step that gains less than a factor 10 means the correction equation is
    // hard for GMRES (a nearby root): the Davidson continuation is cheaper from here
    if (!(rn < 0.1 * last)) throw Err(CCSD_ERR_NOT_CONVERGED, "eigenpair refinement stalled");
    last = rn;
    // GMRES on Op(v) = P (A - w) P M^-1 v, Op(q) = -r, d = P M^-1 q (q accumulated in u)
    auto op = [&](const double* v, double* out) {
      launch_precond(c->vs, c->eps.p, v, z.p, w, c->st);  // z = M^-1 v
      project(z.p);
      transform(z.p, out);
      ++n;
      launch_axpby(dim, -w, z.p, 1.0, out, c->st);
      project(out);
    };
    CUDA_OK(cudaMemsetAsync(u.p, 0, dim * sizeof(double), c->st));
    const double target = std::max(1e-4 * rn, 0.1 * tol);
    double resid = rn;
    for (int cycle = 0; cycle < 4 && resid > target; ++cycle) {
      // v0 = (-r - Op(u)) / beta
      double* v0 = V.p;
      launch_axpby(dim, -1.0, r.p, 0.0, v0, c->st);
      if (cycle > 0) {
        op(u.p, ax.p);
        launch_axpby(dim, -1.0, ax.p, 1.0, v0, c->st);
      }
      const double beta = norm(v0);
      if (!(beta > target)) break;
      launch_axpby(dim, 1.0 / beta, v0, 0.0, v0, c->st);
      std::vector<double> Hm((KR + 1) * KR, 0.0), cs(KR), sn(KR), g(KR + 1, 0.0);
      g[0] = beta;
      int k = 0;
      for (; k < KR; ++k) {
        double* vk1 = V.p + (k + 1) * dim;
        op(V.p + k * dim, vk1);
        // modified Gram-Schmidt against V[0..k], twice
        for (int pass = 0; pass < 2; ++pass) {
          std::vector<double> hcol = gram(c, V.p, dim, k + 1, vk1, dim, 1);
          std::vector<double> coef(k + 1);
          for (int i = 0; i <= k; ++i) {
            Hm[i * KR + k] += hcol[i];
            coef[i] = -hcol[i];
          }
          lincomb(c, V.p, dim, k + 1, coef, vk1, dim, 1, true);
        }
        const double hn = norm(vk1);
        Hm[(k + 1) * KR + k] = hn;
        for (int j = 0; j < k; ++j) {
          const double a = Hm[j * KR + k], b = Hm[(j + 1) * KR + k];
          Hm[j * KR + k] = cs[j] * a + sn[j] * b;
          Hm[(j + 1) * KR + k] = -sn[j] * a + cs[j] * b;
        }
        const double a = Hm[k * KR + k], b = Hm[(k + 1) * KR + k];
        const double den = std::hypot(a, b);
        cs[k] = den > 0 ? a / den : 1.0;
        sn[k] = den > 0 ? b / den : 0.0;
        Hm[k * KR + k] = den;
        Hm[(k + 1) * KR + k] = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        resid = std::fabs(g[k + 1]);
        if (verbose_solvers()) fprintf(stderr, "[refine side %d]   gmres %d.%d: |res| = %.3e\n", side, cycle, k, resid);
        if (hn > 0) launch_axpby(dim, 1.0 / hn, vk1, 0.0, vk1, c->st);
        if (resid <= target || hn == 0.0) {
          ++k;
          break;
        }
      }
      std::vector<double> y(k, 0.0);
      for (int j = k - 1; j >= 0; --j) {
        double s = g[j];
        for (int q = j + 1; q < k; ++q) s -= Hm[j * KR + q] * y[q];
        y[j] = s / Hm[j * KR + j];
      }
      lincomb(c, V.p, dim, k, y, u.p, dim, 1, true);
    }
    // d = P M^-1 u
    launch_precond(c->vs, c->eps.p, u.p, z.p, w, c->st);
    project(z.p);
    launch_axpby(dim, 1.0, z.p, 1.0, x, c->st);
  }
  throw Err(CCSD_ERR_NOT_CONVERGED, "eigenpair refinement did not converge");
}

// normalise R to unit packed norm, largest-magnitude component positive
void normalize_right(ccsd_ctx* c, double* R) {
  std::vector<double> nr = gram(c, R, c->dim, 1, R, c->dim, 1);
  launch_axpby(c->dim, 1.0 / std::sqrt(nr[0]), R, 0.0, R, c->st);
  DevBuf o2(2);
  launch_argmaxabs(c->dim, R, o2.p, c->ex->scratch(1024), c->st);
  double h2[2];
  CUDA_OK(cudaMemcpyAsync(h2, o2.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  if (h2[1] < 0) launch_axpby(c->dim, -1.0, R, 0.0, R, c->st);
}

// right states in c->R with excitation energies w: normalisation, R0 = eta.R / omega
void finish_right(ccsd_ctx* c, const std::vector<double>& w) {
  const int nroots = (int)w.size();
  c->omega = w;
  c->r0.assign(nroots, 0.0);
  for (int k = 0; k < nroots; ++k) {
    normalize_right(c, c->R[k]->p);
    std::vector<double> d = gram(c, c->eta.p, c->dim, 1, c->R[k]->p, c->dim, 1);
    c->r0[k] = d[0] / w[k];
  }
  c->have_right = true;
  c->have_left = false;
  c->dens_k = c->dens_l = -1;
}

// left eigenvectors Lr with excitation energies w: root check against the right
// solve, then biorthonormalisation L_k = sum_m Minv^T[k][m] Lr_m with M[m][l] = <Lr_m|R_l>
void finish_left(ccsd_ctx* c, const std::vector<double>& w, const std::vector<std::unique_ptr<DevBuf>>& Lr) {
  const int nroots = (int)w.size();
  for (int k = 0; k < nroots; ++k)
    if (std::fabs(w[k] - c->omega[k]) > 1e-5 * std::max(1.0, std::fabs(c->omega[k])))
      throw Err(CCSD_ERR_NOT_CONVERGED, "left and right roots differ: root " + std::to_string(k) + " left " +
                                            std::to_string(w[k]) + " right " + std::to_string(c->omega[k]));
  std::vector<double> M(nroots * nroots);
  for (int k = 0; k < nroots; ++k)
    for (int l = 0; l < nroots; ++l) M[k * nroots + l] = gram(c, Lr[k]->p, c->dim, 1, c->R[l]->p, c->dim, 1)[0];
  // the inverse in FP64 on the GPU (subspace.cu)
  std::vector<double> Minv(nroots * nroots);
  {
    DevBuf Md(nroots * nroots), Mi(nroots * nroots), wk((small_inverse_work_bytes(nroots) + 7) / 8), fl(1);
    int flag = 0;
    CUDA_OK(cudaMemcpyAsync(Md.p, M.data(), nroots * nroots * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_small_inverse(nroots, Md.p, Mi.p, (int*)fl.p, wk.p, c->st);
    CUDA_OK(cudaMemcpyAsync(Minv.data(), Mi.p, nroots * nroots * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaMemcpyAsync(&flag, fl.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    if (flag) throw Err(CCSD_ERR_DEGENERATE, "left/right overlap matrix is singular");
  }
  c->L.clear();
  for (int k = 0; k < nroots; ++k) {
    c->L.emplace_back(new DevBuf(c->dim));
    CUDA_OK(cudaMemsetAsync(c->L[k]->p, 0, c->dim * sizeof(double), c->st));
    for (int m = 0; m < nroots; ++m) launch_axpby(c->dim, Minv[k * nroots + m], Lr[m]->p, 1.0, c->L[k]->p, c->st);
  }
  sync(c);
  c->have_left = true;
  c->dens_k = c->dens_l = -1;
}

ccsd_status fail(ccsd_ctx* c, ccsd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

template <typename F>
ccsd_status guarded(ccsd_ctx* c, F&& f) {
  if (!c) return CCSD_ERR_ARG;
  AllocatorScope scope(&c->allocator, c->st);
  try {
    TempScope temps;  // released if f() throws
    f();
    return CCSD_OK;
  } catch (const Err& e) {
    return fail(c, e.code, e.what());
  } catch (const DeviceTimeout& e) {
    return fail(c, CCSD_ERR_TIMEOUT, e.what());
  } catch (const OutOfMemory& e) {
    return fail(c, CCSD_ERR_OOM, e.what());
  } catch (const std::bad_alloc& e) {
    return fail(c, CCSD_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    std::string m = e.what();
    if (m.find("out of memory") != std::string::npos) return fail(c, CCSD_ERR_OOM, m);
    return fail(c, CCSD_ERR_CUDA, m);
  }
}

// copy n doubles from a host or device pointer into a new device buffer
void to_device(ccsd_ctx* c, const double* src, int64_t n, DevBuf& dst) {
  dst.alloc(n);
  CUDA_OK(cudaMemcpyAsync(dst.p, src, n * sizeof(double), cudaMemcpyDefault, c->st));
}

void from_device(ccsd_ctx* c, const double* src, int64_t n, double* dst) {
  CUDA_OK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c->st));
}

// left state k: (l0, L) with L a device vector (k = 0: lambda)
const double* left_vec(ccsd_ctx* c, int k) { return k == 0 ? c->lam.p : c->L[k - 1]->p; }
double omega_of(ccsd_ctx* c, int k) { return k == 0 ? 0.0 : c->omega[k - 1]; }

// ---------------------------------------------------------------------------
// orbital relaxation (Eq. orbitalrelax and the kappa-bar term of Eq. NAC_NC)
// ---------------------------------------------------------------------------

// executor of the Hartree-Fock programs, bound to the handle's integrals (FP64)
Executor& hf_exec(ccsd_ctx* c) {
  if (!c->hx) {
    c->hfp.reset(new HFPrograms);
    build_hf_programs(*c->hfp);
    c->hx.reset(new Executor(c->hfp->g, c->o, c->v, c->naux, 1, c->st));
    c->hx->set_precision(CCSD_PREC_FP64, c->opt.splits);
  }
  Executor& hx = *c->hx;
  hx.set_stream(c->st);
  hx.bind(c->hfp->h, c->h.p);
  hx.bind(c->hfp->B, c->B.p);
  hx.bind(c->hfp->ones_o, c->ones.p);
  return hx;
}

// max |F_ia| of the handle's integrals
double fock_ov_max(ccsd_ctx* c) {
  Executor& hx = hf_exec(c);
  DevBuf f(c->n1);
  hx.bind(c->hfp->F, f.p);
  hx.run(c->hfp->fock);
  return maxabs(c, f.p, c->n1);
}

// Solve J x = rhs for J = dF'_ia/dkappa_jb away from a Hartree-Fock point (not symmetric
// there) by right-preconditioned restarted GMRES(30) on host vectors; J products run in
// the Hartree-Fock programs.  Used for the steps of ccsd_scf.
std::vector<double> hf_solve_general(Executor& hx, const HFPrograms& P, int o, int v, cudaStream_t st,
                                     const std::vector<double>& rhs, const std::vector<double>& eps, double tol,
                                     int maxit) {
  const int64_t m = (int64_t)o * v;
  const int kr = 30;
  DevBuf xd(m), ad(m), fd(m);
  std::vector<double> pre(m);
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) pre[i * v + a] = 1.0 / std::max(eps[o + a] - eps[i], 1e-3);
  auto apply = [&](const std::vector<double>& x) {  // J M^-1 x
    std::vector<double> y(m);
    for (int64_t i = 0; i < m; ++i) y[i] = pre[i] * x[i];
    CUDA_OK(cudaMemcpyAsync(xd.p, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    hx.bind(P.x, xd.p);
    hx.bind(P.AX, ad.p);
    hx.bind(P.F, fd.p);
    hx.run(P.hfA);
    CUDA_OK(cudaMemcpyAsync(y.data(), ad.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    return y;
  };
  auto nrm = [&](const std::vector<double>& a) {
    double s = 0.0;
    for (double q : a) s += q * q;
    return std::sqrt(s);
  };
  std::vector<double> u(m, 0.0);  // solution of J M^-1 u = rhs
  const double bn = nrm(rhs);
  if (bn == 0.0) return u;
  int used = 0;
  while (used < maxit) {
    std::vector<double> r = apply(u);
    ++used;
    for (int64_t i = 0; i < m; ++i) r[i] = rhs[i] - r[i];
    double beta = nrm(r);
    if (beta <= tol * bn) break;
    std::vector<std::vector<double>> V(1, r);
    for (double& q : V[0]) q /= beta;
    std::vector<double> Hm((kr + 1) * kr, 0.0), cs(kr), sn(kr), g(kr + 1, 0.0);
    g[0] = beta;
    int k = 0;
    for (; k < kr && used < maxit; ++k) {
      std::vector<double> w = apply(V[k]);
      ++used;
      for (int j = 0; j <= k; ++j) {
        double h = 0.0;
        for (int64_t i = 0; i < m; ++i) h += w[i] * V[j][i];
        Hm[j * kr + k] = h;
        for (int64_t i = 0; i < m; ++i) w[i] -= h * V[j][i];
      }
      const double hn = nrm(w);
      Hm[(k + 1) * kr + k] = hn;
      for (int j = 0; j < k; ++j) {  // previous rotations
        const double a = Hm[j * kr + k], b = Hm[(j + 1) * kr + k];
        Hm[j * kr + k] = cs[j] * a + sn[j] * b;
        Hm[(j + 1) * kr + k] = -sn[j] * a + cs[j] * b;
      }
      const double a = Hm[k * kr + k], b = Hm[(k + 1) * kr + k];
      const double den = std::hypot(a, b);
      cs[k] = den > 0 ? a / den : 1.0;
      sn[k] = den > 0 ? b / den : 0.0;
      Hm[k * kr + k] = den;
      Hm[(k + 1) * kr + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      if (hn > 0) {
        for (double& q : w) q /= hn;
      }
      V.push_back(w);
      if (std::fabs(g[k + 1]) <= tol * bn || hn == 0.0) {
        ++k;
        break;
      }
    }
    std::vector<double> y(k, 0.0);  // back substitution
    for (int j = k - 1; j >= 0; --j) {
      double s = g[j];
      for (int q = j + 1; q < k; ++q) s -= Hm[j * kr + q] * y[q];
      y[j] = s / Hm[j * kr + j];
    }
    for (int j = 0; j < k; ++j)
      for (int64_t i = 0; i < m; ++i) u[i] += y[j] * V[j][i];
  }
  for (int64_t i = 0; i < m; ++i) u[i] *= pre[i];
  return u;
}

// Solve A^HF x = rhs (A^HF symmetric positive definite at a Hartree-Fock minimum) by
// preconditioned conjugate gradients; A^HF products run in the Hartree-Fock programs,
// the o*v-sized vectors live on the host.  eps gives the preconditioner 1/(e_a - e_i).
std::vector<double> hf_solve(Executor& hx, const HFPrograms& P, int o, int v, cudaStream_t st,
                             const std::vector<double>& rhs, const std::vector<double>& eps, double tol, int maxit) {
  const int64_t m = (int64_t)o * v;
  DevBuf xd(m), ad(m), fd(m);
  auto apply = [&](const std::vector<double>& x) {
    CUDA_OK(cudaMemcpyAsync(xd.p, x.data(), m * sizeof(double), cudaMemcpyHostToDevice, st));
    hx.bind(P.x, xd.p);
    hx.bind(P.AX, ad.p);
    hx.bind(P.F, fd.p);
    hx.run(P.hfA);
    std::vector<double> y(m);
    CUDA_OK(cudaMemcpyAsync(y.data(), ad.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
    return y;
  };
  auto dot = [&](const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
  };
  std::vector<double> pre(m);
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) pre[i * v + a] = 1.0 / std::max(eps[o + a] - eps[i], 1e-3);
  std::vector<double> x(m, 0.0), r = rhs, z(m), p(m);
  const double bn = std::sqrt(dot(rhs, rhs));
  if (bn == 0.0) return x;
  for (int64_t i = 0; i < m; ++i) z[i] = pre[i] * r[i];
  p = z;
  double rz = dot(r, z);
  for (int it = 0; it < maxit; ++it) {
    std::vector<double> Ap = apply(p);
    const double pAp = dot(p, Ap);
    if (!(pAp > 0.0)) throw Err(CCSD_ERR_NOT_HF, "the Hartree-Fock Hessian is not positive definite");
    const double alpha = rz / pAp;
    for (int64_t i = 0; i < m; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    if (std::sqrt(dot(r, r)) <= tol * bn) return x;
    for (int64_t i = 0; i < m; ++i) z[i] = pre[i] * r[i];
    const double rz1 = dot(r, z);
    for (int64_t i = 0; i < m; ++i) p[i] = z[i] + (rz1 / rz) * p[i];
    rz = rz1;
  }
  throw Err(CCSD_ERR_NOT_CONVERGED, "orbital-response equations not converged");
}

// One-electron transition density D_pq = <psi_k^L| E_pq |psi_l^R> (n x n, device), the
// derivative of <psi_k^L|H|psi_l^R> with respect to h_pq at fixed states.  Over the
// reference, singles and doubles,
//   <psi^L|H|psi^R> = E (l0 r0 + L.R) + l0 eta.R + L.(r0 Omega + A R) + w.Omega,
// with w_k = <L| tau_k R_1 |HF> (singles of R carried by one more excitation), so D is
// the h-part of the density programs with seeds z = r0 L + w, g = L, g0 = l0 along R,
// plus (l0 r0 + L.R) times the energy's own density.
void transition_density(ccsd_ctx* c, int k, int l, double* D) {
  const int64_t dim = c->dim, nn = (int64_t)c->n * c->n, nz = (int64_t)c->naux * nn;
  auto& P = c->P;
  Executor& ex = *c->ex;
  const double l0 = (k == 0) ? 1.0 : 0.0;
  const double* L = left_vec(c, k);
  DevBuf WL(dim), Zs(nz), e0(1), D2(nn);
  launch_weight(c->vs, L, WL.p, 1, dim, c->st);
  if (l == 0) {  // r0 = 1, R = 0: d/dh of l0 E + L.Omega
    CUDA_OK(cudaMemcpyAsync(e0.p, &l0, sizeof(double), cudaMemcpyHostToDevice, c->st));
    ex.set_nvec(1);
    ex.bind(P.eZ1, WL.p);
    ex.bind(P.eZ2, WL.p + c->n1);
    ex.bind(P.eE, e0.p);
    ex.bind(P.eH, D);
    ex.bind(P.eB, Zs.p);
    ex.run(P.dens0);
    sync(c);
    return;
  }
  const double r0 = c->r0[l - 1];
  const double* R = c->R[l - 1]->p;
  const double cE = l0 * r0 + gram(c, L, dim, 1, R, dim, 1)[0];
  DevBuf R1(dim), w(dim), z(dim), Wz(dim), s0(1), zero(dim);
  CUDA_OK(cudaMemsetAsync(R1.p, 0, dim * sizeof(double), c->st));
  CUDA_OK(cudaMemcpyAsync(R1.p, R, c->n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  launch_tau_expectation(c->vs, 0.0, L, R1.p, w.p, c->st);
  CUDA_OK(cudaMemsetAsync(w.p + c->n1, 0, (dim - c->n1) * sizeof(double), c->st));
  launch_axpby(dim, r0, L, 0.0, z.p, c->st);
  launch_axpby(dim, 1.0, w.p, 1.0, z.p, c->st);
  launch_weight(c->vs, z.p, Wz.p, 1, dim, c->st);
  CUDA_OK(cudaMemcpyAsync(s0.p, &l0, sizeof(double), cudaMemcpyHostToDevice, c->st));
  ex.set_nvec(1);
  ex.bind(P.dZ1, Wz.p);
  ex.bind(P.dZ2, Wz.p + c->n1);
  ex.bind(P.dG1, WL.p);
  ex.bind(P.dG2, WL.p + c->n1);
  ex.bind(P.dG0, s0.p);
  ex.bind(P.dR1, const_cast<double*>(R));
  ex.bind(P.dR2, const_cast<double*>(R) + c->n1);
  ex.bind(P.dH, D);
  ex.bind(P.dB, Zs.p);
  ex.run(P.dens1);
  // + cE dE/dh
  CUDA_OK(cudaMemsetAsync(zero.p, 0, dim * sizeof(double), c->st));
  CUDA_OK(cudaMemcpyAsync(e0.p, &cE, sizeof(double), cudaMemcpyHostToDevice, c->st));
  ex.bind(P.eZ1, zero.p);
  ex.bind(P.eZ2, zero.p + c->n1);
  ex.bind(P.eE, e0.p);
  ex.bind(P.eH, D2.p);
  ex.bind(P.eB, Zs.p);
  ex.run(P.dens0);
  launch_axpby(nn, 1.0, D2.p, 1.0, D, c->st);
  sync(c);
}

// With the condition densities of the pair in Dd, Zd: k-eta, kappa-bar, and the
// kappa-bar densities added to Dd, Zd (so that the coupling contraction carries
// kappa-bar_ai F^q_ai).
// overlap = false (state-energy gradients): the Lagrangian has no overlap term, so k-eta is
// the condition part alone.
void add_orbital_relaxation(ccsd_ctx* c, int k, int l, bool overlap = true) {
  const int o = c->o, v = c->v, n = c->n;
  const int64_t nn = (int64_t)n * n, nz = (int64_t)c->naux * nn, m = (int64_t)o * v;
  PrecScope fp64(c, fp64_prec(c));
  DevBuf Dt(nn);
  if (overlap)
    transition_density(c, k, l, Dt.p);
  else
    CUDA_OK(cudaMemsetAsync(Dt.p, 0, nn * sizeof(double), c->st));
  Executor& hx = hf_exec(c);
  const HFPrograms& P = *c->hfp;
  // condition part of k-eta: the adjoint of the rotation map applied to (D, Z)
  DevBuf xb(m);
  hx.bind(P.dD, c->Dd.p);
  hx.bind(P.dZ, c->Zd.p);
  hx.bind(P.xbar, xb.p);
  hx.run(P.rotT);
  std::vector<double> ke(m), Dh(nn), eps(n);
  CUDA_OK(cudaMemcpyAsync(ke.data(), xb.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(cudaMemcpyAsync(Dh.data(), Dt.p, nn * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(cudaMemcpyAsync(eps.data(), c->eps.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  // overlap part: D_ai - D_ia of the transition density
  for (int i = 0; i < o; ++i)
    for (int a = 0; a < v; ++a) ke[i * v + a] += Dh[(int64_t)(o + a) * n + i] - Dh[(int64_t)i * n + o + a];
  // kappa-bar^T A^HF = -k-eta^T, A^HF symmetric
  std::vector<double> rhs(m);
  for (int64_t i = 0; i < m; ++i) rhs[i] = -ke[i];
  c->kbar = hf_solve(hx, P, o, v, c->st, rhs, eps, 1e-13, 500);
  // densities of kappa-bar.F, added to the pair's densities
  DevBuf kb(m), kH(nn), kB(nz), fd(m);
  CUDA_OK(cudaMemcpyAsync(kb.p, c->kbar.data(), m * sizeof(double), cudaMemcpyHostToDevice, c->st));
  hx.bind(P.kbar, kb.p);
  hx.bind(P.F, fd.p);
  hx.bind(P.kH, kH.p);
  hx.bind(P.kB, kB.p);
  hx.run(P.kdens);
  launch_axpby(nn, 1.0, kH.p, 1.0, c->Dd.p, c->st);
  launch_axpby(nz, 1.0, kB.p, 1.0, c->Zd.p, c->st);
  sync(c);
}

// Start of a multiplier solve x^T A = -rhs^T: the Jacobi step x = -rhs/D, its doubles
// corrected, when the handle has a multiplier model, by the model's prediction from the
// per-element features (x_2, D, |(ia|jb)|).
void multiplier_start(ccsd_ctx* c, const double* rhs, double* x) {
  launch_precond(c->vs, c->eps.p, rhs, x, 0.0, c->st);
  launch_axpby(c->dim, 0.0, x, -1.0, x, c->st);
  if (!c->mult_model.p) return;
  const int64_t n2 = c->dim - c->n1;
  DevBuf X((n2 * 3 + 1) / 2), delta((n2 + 1) / 2);
  const double* gov = c->ex->ptr(c->P.cp.g.id("Govov"));
  mlp::features(gov, c->eps.p, c->o, c->v, (float*)X.p, c->st, x + c->n1);
  mlp::predict((const float*)c->mult_model.p, (const float*)X.p, n2, (float*)delta.p, c->st);
  mlp::add_delta(x + c->n1, (const float*)delta.p, n2, c->st);
  sync(c);
}

void compute_densities(ccsd_ctx* c, int k, int l) {
  const int nr = (int)c->omega.size();
  if (k < 0 || l < 0 || k == l) throw Err(CCSD_ERR_ARG, "state indices must differ and be >= 0");
  if (k > nr || l > nr) throw Err(CCSD_ERR_ARG, "state index beyond the solved roots");
  if ((k > 0 || l > 0) && !(c->have_right && c->have_left)) throw Err(CCSD_ERR_STATE, "EOM states not solved");
  if (c->dens_k == k && c->dens_l == l) return;
  ensure_cache(c);
  const int64_t dim = c->dim;
  auto& P = c->P;
  Executor& ex = *c->ex;
  if (!c->Dd.p) c->Dd.alloc((int64_t)c->n * c->n);
  if (!c->Zd.p) c->Zd.alloc((int64_t)c->naux * c->n * c->n);
  DevBuf zeta(dim), Wz(dim);
  if (l == 0) {
    // zeta = L_k / (E_0 - E_k) = -L_k / omega_k  (Eqs. for the ground-state right state)
    launch_axpby(dim, -1.0 / c->omega[k - 1], c->L[k - 1]->p, 0.0, zeta.p, c->st);
    launch_weight(c->vs, zeta.p, Wz.p, 1, dim, c->st);
    DevBuf e0(1);
    CUDA_OK(cudaMemsetAsync(e0.p, 0, sizeof(double), c->st));
    ex.set_nvec(1);
    ex.bind(P.eZ1, Wz.p);
    ex.bind(P.eZ2, Wz.p + c->n1);
    ex.bind(P.eE, e0.p);
    ex.bind(P.eH, c->Dd.p);
    ex.bind(P.eB, c->Zd.p);
    PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
    ex.run(P.dens0);
  } else {
    double dw = omega_of(c, l) - omega_of(c, k);
    if (std::fabs(dw) < c->opt.tol_degen) throw Err(CCSD_ERR_DEGENERATE, "omega_l - omega_k below threshold");
    const double l0 = (k == 0) ? 1.0 : 0.0;
    const double g0 = l0 / dw;
    const double* Rl = c->R[l - 1]->p;
    const double r0 = c->r0[l - 1];
    DevBuf gam(dim), teta(dim), hv(dim), Wg(dim), s0(1);
    launch_axpby(dim, 1.0 / dw, left_vec(c, k), 0.0, gam.p, c->st);
    // t-eta = <L_k|tau|R_l> + d^2(g0 E + gamma.Omega)/dt^2 R_l
    launch_tau_expectation(c->vs, r0, left_vec(c, k), Rl, teta.p, c->st);
    {
      PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
      hess_right(c, g0, gam.p, Rl, hv.p);
    }
    launch_axpby(dim, 1.0, hv.p, 1.0, teta.p, c->st);
    // zeta^T A = -t-eta^T (Eq. amplituderelax)
    multiplier_start(c, teta.p, zeta.p);
    c->iters_zeta = solve_left_refined(c, teta.p, zeta.p, c->opt.tol_lin);
    launch_weight(c->vs, zeta.p, Wz.p, 1, dim, c->st);
    launch_weight(c->vs, gam.p, Wg.p, 1, dim, c->st);
    CUDA_OK(cudaMemcpyAsync(s0.p, &g0, sizeof(double), cudaMemcpyHostToDevice, c->st));
    ensure_cache(c);
    ex.set_nvec(1);
    ex.bind(P.dZ1, Wz.p);
    ex.bind(P.dZ2, Wz.p + c->n1);
    ex.bind(P.dG1, Wg.p);
    ex.bind(P.dG2, Wg.p + c->n1);
    ex.bind(P.dG0, s0.p);
    ex.bind(P.dR1, const_cast<double*>(Rl));
    ex.bind(P.dR2, const_cast<double*>(Rl) + c->n1);
    ex.bind(P.dH, c->Dd.p);
    ex.bind(P.dB, c->Zd.p);
    PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
    ex.run(P.dens1);
  }
  sync(c);
  if (c->opt.relax_orbitals) add_orbital_relaxation(c, k, l);
  c->dens_k = k;
  c->dens_l = l;
}

// dens_l value marking that Dd, Zd hold the state-energy gradient densities of state dens_k
constexpr int kGradientDensities = -2;

// Densities D = dL/dh, Z = dL/dB of the energy Lagrangian of state k at the solved
// amplitudes and multipliers (the Lagrangian construction of the paper with the state
// energy in place of the overlap):
//   k = 0:  L = E + lambda.Omega                         (lambda^T A = -eta^T)
//   k >= 1: L = E + lambda.Omega + L_k.(A R_k) + zeta.Omega, zeta^T A = -(F(L_k) R_k)^T,
// since E_k = E_0 + omega_k and omega_k = L_k.(A R_k) is stationary in the biorthonormal
// L_k, R_k (L_k.R_k = 1, l_0 = 0), so only its amplitude dependence needs a multiplier.
// Relaxed orbitals add kappa-bar from kappa-bar^T A^HF = -k-eta^T (no overlap term).
void compute_gradient_densities(ccsd_ctx* c, int k) {
  const int nr = (int)c->omega.size();
  if (k < 0 || k > nr) throw Err(CCSD_ERR_ARG, "state index beyond the solved roots");
  if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
  if (k > 0 && !(c->have_right && c->have_left)) throw Err(CCSD_ERR_STATE, "EOM states not solved");
  if (c->dens_k == k && c->dens_l == kGradientDensities) return;
  c->dens_k = c->dens_l = -1;
  ensure_cache(c);
  const int64_t dim = c->dim, nn = (int64_t)c->n * c->n, nz = (int64_t)c->naux * nn;
  auto& P = c->P;
  Executor& ex = *c->ex;
  if (!c->Dd.p) c->Dd.alloc(nn);
  if (!c->Zd.p) c->Zd.alloc(nz);
  // E + lambda.Omega
  {
    DevBuf Wl(dim), e1(1);
    const double one = 1.0;
    launch_weight(c->vs, c->lam.p, Wl.p, 1, dim, c->st);
    CUDA_OK(cudaMemcpyAsync(e1.p, &one, sizeof(double), cudaMemcpyHostToDevice, c->st));
    ex.set_nvec(1);
    ex.bind(P.eZ1, Wl.p);
    ex.bind(P.eZ2, Wl.p + c->n1);
    ex.bind(P.eE, e1.p);
    ex.bind(P.eH, c->Dd.p);
    ex.bind(P.eB, c->Zd.p);
    PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
    ex.run(P.dens0);
    sync(c);
  }
  if (k > 0) {
    const double* Lk = c->L[k - 1]->p;
    const double* Rk = c->R[k - 1]->p;
    DevBuf hv(dim), zeta(dim), Wz(dim), WL(dim), s0(1), D2(nn), Z2(nz);
    {
      PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
      hess_right(c, 0.0, Lk, Rk, hv.p);
    }
    // zeta^T A = -(F(L_k) R_k)^T
    multiplier_start(c, hv.p, zeta.p);
    c->iters_zeta = solve_left_refined(c, hv.p, zeta.p, c->opt.tol_lin);
    launch_weight(c->vs, zeta.p, Wz.p, 1, dim, c->st);
    launch_weight(c->vs, Lk, WL.p, 1, dim, c->st);
    CUDA_OK(cudaMemsetAsync(s0.p, 0, sizeof(double), c->st));
    ensure_cache(c);
    ex.set_nvec(1);
    ex.bind(P.dZ1, Wz.p);
    ex.bind(P.dZ2, Wz.p + c->n1);
    ex.bind(P.dG1, WL.p);
    ex.bind(P.dG2, WL.p + c->n1);
    ex.bind(P.dG0, s0.p);
    ex.bind(P.dR1, const_cast<double*>(Rk));
    ex.bind(P.dR2, const_cast<double*>(Rk) + c->n1);
    ex.bind(P.dH, D2.p);
    ex.bind(P.dB, Z2.p);
    {
      PrecScope p(c, refining(c) ? fp64_prec(c) : ex.precision());
      ex.run(P.dens1);
    }
    launch_axpby(nn, 1.0, D2.p, 1.0, c->Dd.p, c->st);
    launch_axpby(nz, 1.0, Z2.p, 1.0, c->Zd.p, c->st);
    sync(c);
  }
  if (c->opt.relax_orbitals) add_orbital_relaxation(c, k, k, false);
  c->dens_k = k;
  c->dens_l = kGradientDensities;
}

// F[d] = <Dd, dh[d]> + <Zd, dB[d]> for the densities the handle holds (host or device directions)
void contract_densities(ccsd_ctx* c, int ndir, const double* dh, const double* dB, double* F) {
  const int64_t nn = (int64_t)c->n * c->n, nb = (int64_t)c->naux * nn;
  DevBuf out(2), tmp;
  bool hdev = is_device_ptr(dh), bdev = is_device_ptr(dB);
  double* work = c->ex->scratch(1024);
  for (int d = 0; d < ndir; ++d) {
    double fh, fb;
    const double* hp = dh + d * nn;
    if (!hdev) {
      to_device(c, hp, nn, tmp);
      hp = tmp.p;
    }
    launch_dot(nn, c->Dd.p, hp, out.p, work, c->st);
    CUDA_OK(cudaMemcpyAsync(&fh, out.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    const double* bp = dB + d * nb;
    if (!bdev) {
      to_device(c, bp, nb, tmp);
      bp = tmp.p;
    }
    launch_dot(nb, c->Zd.p, bp, out.p, work, c->st);
    CUDA_OK(cudaMemcpyAsync(&fb, out.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    F[d] = fh + fb;
  }
}

}  // namespace

extern "C" {

void ccsd_default_options(ccsd_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = CCSD_PREC_FP64;
  opt->splits = 3;
  opt->relax_orbitals = 0;
  opt->tol_res = 1e-10;
  opt->tol_eom = 1e-7;
  opt->tol_lin = 1e-9;
  opt->tol_degen = 1e-8;
  opt->max_iter = 100;
  opt->diis_dim = 8;
  opt->davidson_block = 8;
  opt->davidson_max_sub = 48;
  opt->guess = CCSD_GUESS_MP2;
  opt->stream = nullptr;
  opt->tc_min_flops = 1.0e8;
  opt->refine = 1;
  opt->tol_switch = 1e-6;
  opt->autotune = 0;
  opt->fp64_tc = 1;
}

const char* ccsd_strerror(ccsd_status s) {
  switch (s) {
    case CCSD_OK: return "ok";
    case CCSD_ERR_ARG: return "invalid argument";
    case CCSD_ERR_OOM: return "out of device memory";
    case CCSD_ERR_CUDA: return "CUDA error";
    case CCSD_ERR_STATE: return "prerequisite call missing";
    case CCSD_ERR_NOT_CONVERGED: return "not converged";
    case CCSD_ERR_COMPLEX_ROOT: return "complex EOM root";
    case CCSD_ERR_DEGENERATE: return "degenerate states";
    case CCSD_ERR_NOT_HF: return "reference is not Hartree-Fock";
    case CCSD_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* ccsd_last_error(ccsd_handle h) {
  if (h) return h->err.c_str();
  return g_last_error.empty() ? "no error recorded" : g_last_error.c_str();
}

ccsd_status ccsd_create(const double* eps, const double* h, const double* B, int o, int v, int naux,
                        const ccsd_options* opt, ccsd_handle* out) {
  if (!out) return CCSD_ERR_ARG;
  *out = nullptr;
  if (!eps || !h || !B || o < 1 || v < 1 || naux < 1) return CCSD_ERR_ARG;
  ccsd_ctx* c = new (std::nothrow) ccsd_ctx();
  if (!c) return CCSD_ERR_OOM;
  if (opt)
    c->opt = *opt;
  else
    ccsd_default_options(&c->opt);
  if ((c->opt.alloc != nullptr) != (c->opt.free != nullptr)) {
    delete c;
    return CCSD_ERR_ARG;
  }
  c->allocator.alloc = c->opt.alloc;
  c->allocator.free = c->opt.free;
  c->allocator.ctx = c->opt.alloc_ctx;
  c->st = (cudaStream_t)c->opt.stream;
  if ((c->opt.relax_orbitals != 0 && c->opt.relax_orbitals != 1) ||
      (c->opt.precision != CCSD_PREC_FP64 && c->opt.precision != CCSD_PREC_MIXED &&
       c->opt.precision != CCSD_PREC_FP64_TC)) {
    delete c;
    return CCSD_ERR_ARG;
  }
  ccsd_status s = guarded(c, [&] {
    c->o = o;
    c->v = v;
    c->naux = naux;
    c->n = o + v;
    c->vs = VecShape{o, v};
    c->n1 = (int64_t)o * v;
    c->dim = c->vs.dim();
    c->st = (cudaStream_t)c->opt.stream;
    CUDA_OK(cudaGetDevice(&c->device));
    // symmetry of the inputs
    {
      const int64_t n = c->n;
      std::vector<double> hh(n * n), Bh((int64_t)naux * n * n);
      CUDA_OK(cudaMemcpy(hh.data(), h, n * n * sizeof(double), cudaMemcpyDefault));
      CUDA_OK(cudaMemcpy(Bh.data(), B, (int64_t)naux * n * n * sizeof(double), cudaMemcpyDefault));
      double scale = 1e-300, asym = 0.0;
      for (int64_t J = 0; J <= naux; ++J) {
        const double* m = (J == naux) ? hh.data() : Bh.data() + J * n * n;
        for (int64_t p = 0; p < n; ++p)
          for (int64_t q = 0; q < p; ++q) {
            asym = std::max(asym, std::fabs(m[p * n + q] - m[q * n + p]));
            scale = std::max(scale, std::fabs(m[p * n + q]));
          }
      }
      for (double x : hh)
        if (!std::isfinite(x)) throw Err(CCSD_ERR_ARG, "non-finite h");
      for (double x : Bh)
        if (!std::isfinite(x)) throw Err(CCSD_ERR_ARG, "non-finite B");
      if (asym > 1e-10 * std::max(1.0, scale)) throw Err(CCSD_ERR_ARG, "h or B is not symmetric in pq");
    }
    to_device(c, eps, c->n, c->eps);
    to_device(c, h, (int64_t)c->n * c->n, c->h);
    to_device(c, B, (int64_t)naux * c->n * c->n, c->B);
    c->t.alloc(c->dim);
    c->lam.alloc(c->dim);
    c->eta.alloc(c->dim);
    c->escal.alloc(16);
    c->seedE.alloc(16);
    c->gsc.alloc(16);
    CUDA_OK(cudaMemsetAsync(c->t.p, 0, c->dim * sizeof(double), c->st));
    std::vector<double> ones(o, 1.0);
    c->ones.alloc(o);
    CUDA_OK(cudaMemcpyAsync(c->ones.p, ones.data(), o * sizeof(double), cudaMemcpyHostToDevice, c->st));
    build_programs(c->P);
    auto& cp = c->P.cp;
    c->ex.reset(new Executor(cp.g, o, v, naux, 16, c->st));
    Executor& ex = *c->ex;
    ex.set_precision(c->opt.precision, c->opt.splits);
    ex.tc_min_flops = c->opt.tc_min_flops;
    ex.autotune = c->opt.autotune;
    ex.bind(cp.h, c->h.p);
    ex.bind(cp.B, c->B.p);
    ex.bind(cp.ones_o, c->ones.p);
    // persistent storage for everything the forward program writes (primal cache)
    for (const Op& op : cp.fwd) {
      int t = op.out.t;
      if (t == cp.O1 || t == cp.O2 || t == cp.E) continue;
      ex.alloc_persistent(t);
    }
    ex.ladder_w_ = cp.g.id("W");
    ex.const_tensors = {cp.h, cp.B, cp.ones_o};
    for (const Op& op : cp.fwd_const) ex.const_tensors.insert(op.out.t);
    // the amplitudes and the intermediates computed from them change only when the
    // forward program runs again (forward() drops their cached slices first)
    ex.frozen_tensors = {cp.t1, cp.t2};
    for (const Op& op : cp.fwd_t)
      if (op.out.t != cp.O1 && op.out.t != cp.O2 && op.out.t != cp.E) ex.frozen_tensors.insert(op.out.t);
    {
      // under FP64 refinement the Hamiltonian-only intermediates are built in FP64,
      // so that the refined equations are exactly the FP64 ones
      const int p0 = ex.precision();
      if (refining(c)) ex.set_precision(fp64_prec(c), c->opt.splits);
      ex.run(cp.fwd_const);
      ex.set_precision(p0, c->opt.splits);
    }
    sync(c);
    // orbital relaxation needs Hartree-Fock orbitals: F_ai = 0
    if (c->opt.relax_orbitals) {
      const double f = fock_ov_max(c);
      if (!(f < 1e-8))
        throw Err(CCSD_ERR_NOT_HF, "relax_orbitals needs Hartree-Fock orbitals: max |F_ia| = " + std::to_string(f));
    }
  });
  if (s != CCSD_OK) {
    delete c;
    return s;
  }
  *out = c;
  return CCSD_OK;
}

void ccsd_destroy(ccsd_handle h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  AllocatorScope scope(&h->allocator, h->st);  // the handle's memory goes back to its allocator
  delete h;
}

ccsd_status ccsd_residual(ccsd_handle c, const double* t, double* omega, double* e) {
  return guarded(c, [&] {
    if (!t || !omega) throw Err(CCSD_ERR_ARG, "null pointer");
    DevBuf td, od(c->dim);
    to_device(c, t, c->dim, td);
    double en = forward(c, td.p, od.p);
    c->cache_at_t = false;
    from_device(c, od.p, c->dim, omega);
    sync(c);
    if (e) *e = en;
  });
}

ccsd_status ccsd_solve_ground(ccsd_handle c, double* e_ccsd, int* iters) {
  return guarded(c, [&] {
    const int64_t dim = c->dim;
    DevBuf om(dim), tn(dim);
    Diis diis(c, c->opt.diis_dim);
    CUDA_OK(cudaMemsetAsync(c->t.p, 0, dim * sizeof(double), c->st));
    c->have_ground = c->have_right = c->have_left = false;
    c->dens_k = c->dens_l = -1;
    int it = 1;
    double e = 0.0;
    const bool refine = refining(c);
    // mixed phase stops at tol_switch (or when it stalls); refinement follows
    const double tol1 = refine ? std::max(c->opt.tol_res, c->opt.tol_switch) : c->opt.tol_res;
    double best = 1e300;
    int since_best = 0;
    for (;; ++it) {
      if (it > c->opt.max_iter) throw Err(CCSD_ERR_NOT_CONVERGED, "ground state not converged");
      e = forward(c, c->t.p, om.p);
      double err = maxabs(c, om.p, dim);
      if (!std::isfinite(err) || !std::isfinite(e)) throw Err(CCSD_ERR_NOT_CONVERGED, "ground state diverged");
      if (err < tol1) break;
      if (err < 0.5 * best) {
        best = err;
        since_best = 0;
      } else if (refine && ++since_best >= 6 && err < 1e3 * tol1) {
        break;  // at the mixed-precision floor
      }
      launch_precond(c->vs, c->eps.p, om.p, tn.p, 0.0, c->st);
      launch_axpby(dim, 1.0, c->t.p, -1.0, tn.p, c->st);  // tn = t - Omega/D
      if (it == 1 && c->guess_model.p) {
        // learned start: t2 = t_MP2 + MLP(features) (t_MP2 = -Omega_2(0)/D is tn's doubles)
        const int64_t n2 = dim - c->n1;
        DevBuf X((n2 * 3 + 1) / 2), delta((n2 + 1) / 2);
        const double* gov = c->ex->ptr(c->P.cp.g.id("Govov"));
        mlp::features(gov, c->eps.p, c->o, c->v, (float*)X.p, c->st);
        mlp::predict((const float*)c->guess_model.p, (const float*)X.p, n2, (float*)delta.p, c->st);
        mlp::add_delta(tn.p + c->n1, (const float*)delta.p, n2, c->st);
        sync(c);
      }
      diis.step(tn.p, om.p, c->t.p);
      c->cache_at_t = false;
    }
    if (refine) {
      // Newton-type defect correction: Omega_64(t) in FP64, A d = -Omega_64 solved
      // with mixed-precision right transforms at t, t += d
      DevBuf d(dim);
      c->have_ground = true;  // the transforms below need the amplitudes in place
      for (int outer = 0;; ++outer) {
        if (outer >= 20) throw Err(CCSD_ERR_NOT_CONVERGED, "FP64 refinement of the ground state did not converge");
        {
          PrecScope fp64(c, fp64_prec(c));
          e = forward(c, c->t.p, om.p);
        }
        ++it;
        double err = maxabs(c, om.p, dim);
        if (!std::isfinite(err)) throw Err(CCSD_ERR_NOT_CONVERGED, "ground state refinement diverged");
        if (err < c->opt.tol_res) break;
        launch_precond(c->vs, c->eps.p, om.p, d.p, 0.0, c->st);
        launch_axpby(dim, 0.0, d.p, -1.0, d.p, c->st);
        it += solve_right_linear(c, om.p, d.p, std::max(1e-3 * err, 0.1 * c->opt.tol_res), c->opt.max_iter);
        launch_axpby(dim, 1.0, d.p, 1.0, c->t.p, c->st);
        c->cache_at_t = false;
      }
    }
    c->e_ccsd = e;
    c->have_ground = true;
    // eta = dE/dt (FP64) and the ground-state multipliers lambda^T A = -eta^T
    DevBuf zero(dim);
    CUDA_OK(cudaMemsetAsync(zero.p, 0, dim * sizeof(double), c->st));
    {
      PrecScope p(c, refine ? fp64_prec(c) : c->ex->precision());
      left_block(c, zero.p, c->eta.p, 1, 1.0);
    }
    multiplier_start(c, c->eta.p, c->lam.p);
    c->iters_lambda = solve_left_refined(c, c->eta.p, c->lam.p, c->opt.tol_lin);
    c->iters_ground = it;
    if (e_ccsd) *e_ccsd = e;
    if (iters) *iters = it;
  });
}

ccsd_status eom_solve_right(ccsd_handle c, int nroots, double* omega, int* iters) {
  return guarded(c, [&] {
    if (nroots < 1 || nroots > c->n1) throw Err(CCSD_ERR_ARG, "bad nroots");
    if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
    std::vector<double> w;
    int it = davidson_refined(c, 0, nroots, w, c->R);
    finish_right(c, w);
    if (omega) std::copy(w.begin(), w.end(), omega);
    if (iters) *iters = it;
  });
}

ccsd_status eom_solve_left(ccsd_handle c, int nroots, double* omega, int* iters) {
  return guarded(c, [&] {
    if (!c->have_right) throw Err(CCSD_ERR_STATE, "eom_solve_right first");
    if (nroots != (int)c->omega.size()) throw Err(CCSD_ERR_ARG, "nroots differs from the right solve");
    std::vector<double> w;
    std::vector<std::unique_ptr<DevBuf>> Lr;
    // the right eigenvectors start the left solve: same roots, close vectors
    int it = davidson_refined(c, 1, nroots, w, Lr, &c->R, &c->omega);
    finish_left(c, w, Lr);
    if (omega) std::copy(w.begin(), w.end(), omega);
    if (iters) *iters = it;
  });
}

ccsd_status ccsd_jacobian_transform(ccsd_handle c, int side, int nvec, const double* x, double* y) {
  return guarded(c, [&] {
    if ((side != 0 && side != 1) || nvec < 1 || !x || !y) throw Err(CCSD_ERR_ARG, "bad arguments");
    const int64_t dim = c->dim;
    const double* xp = x;
    double* yp = y;
    bool xdev = is_device_ptr(x), ydev = is_device_ptr(y);
    if (!xdev) {
      if (c->stage_x.n < nvec * dim) c->stage_x.alloc(nvec * dim);
      CUDA_OK(cudaMemcpyAsync(c->stage_x.p, x, nvec * dim * sizeof(double), cudaMemcpyDefault, c->st));
      xp = c->stage_x.p;
    }
    if (!ydev) {
      if (c->stage_y.n < nvec * dim) c->stage_y.alloc(nvec * dim);
      yp = c->stage_y.p;
    }
    const int block = 16;
    for (int s = 0; s < nvec; s += block) {
      int nb = std::min(block, nvec - s);
      if (side == 0)
        right_block(c, xp + s * dim, yp + s * dim, nb);
      else
        left_block(c, xp + s * dim, yp + s * dim, nb);
    }
    if (!ydev) from_device(c, yp, nvec * dim, y);
    sync(c);
  });
}

ccsd_status ccsd_set_amplitudes(ccsd_handle c, const double* t, const double* lambda, double* e) {
  return guarded(c, [&] {
    if (!t) throw Err(CCSD_ERR_ARG, "null amplitudes");
    const int64_t dim = c->dim;
    CUDA_OK(cudaMemcpyAsync(c->t.p, t, dim * sizeof(double), cudaMemcpyDefault, c->st));
    c->have_ground = c->have_right = c->have_left = false;
    c->dens_k = c->dens_l = -1;
    DevBuf om(dim);
    double en = forward(c, c->t.p, om.p);
    c->e_ccsd = en;
    c->have_ground = true;
    DevBuf zero(dim);
    CUDA_OK(cudaMemsetAsync(zero.p, 0, dim * sizeof(double), c->st));
    {
      PrecScope p(c, refining(c) ? fp64_prec(c) : c->ex->precision());
      left_block(c, zero.p, c->eta.p, 1, 1.0);
    }
    if (lambda) {
      CUDA_OK(cudaMemcpyAsync(c->lam.p, lambda, dim * sizeof(double), cudaMemcpyDefault, c->st));
    } else {
      multiplier_start(c, c->eta.p, c->lam.p);
      c->iters_lambda = solve_left_refined(c, c->eta.p, c->lam.p, c->opt.tol_lin);
    }
    sync(c);
    if (e) *e = en;
  });
}

ccsd_status ccsd_get_amplitudes(ccsd_handle c, double* t, double* lambda) {
  return guarded(c, [&] {
    if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
    if (t) from_device(c, c->t.p, c->dim, t);
    if (lambda) from_device(c, c->lam.p, c->dim, lambda);
    sync(c);
  });
}

ccsd_status ccsd_get_states(ccsd_handle c, int nroots, double* r0, double* right, double* left) {
  return guarded(c, [&] {
    if (!c->have_right) throw Err(CCSD_ERR_STATE, "EOM states not solved");
    if (nroots < 1 || nroots > (int)c->omega.size()) throw Err(CCSD_ERR_ARG, "bad nroots");
    if (left && !c->have_left) throw Err(CCSD_ERR_STATE, "left states not solved");
    for (int k = 0; k < nroots; ++k) {
      if (r0) r0[k] = c->r0[k];
      if (right) from_device(c, c->R[k]->p, c->dim, right + k * c->dim);
      if (left) from_device(c, c->L[k]->p, c->dim, left + k * c->dim);
    }
    sync(c);
  });
}

ccsd_status ccsd_coupling_densities(ccsd_handle c, int k, int l, double* D, double* Z) {
  return guarded(c, [&] {
    compute_densities(c, k, l);
    if (D) from_device(c, c->Dd.p, (int64_t)c->n * c->n, D);
    if (Z) from_device(c, c->Zd.p, (int64_t)c->naux * c->n * c->n, Z);
    sync(c);
  });
}

ccsd_status ccsd_derivative_coupling(ccsd_handle c, int k, int l, int ndir, const double* dh, const double* dB,
                                     double* F) {
  return guarded(c, [&] {
    if (ndir < 1 || !dh || !dB || !F) throw Err(CCSD_ERR_ARG, "bad arguments");
    compute_densities(c, k, l);
    contract_densities(c, ndir, dh, dB, F);
  });
}

}  // extern "C"

namespace {
// checks of the state indices of a transition density (k, l) and the states it needs
void check_pair(ccsd_ctx* c, int k, int l) {
  const int nr = (int)c->omega.size();
  if (k < 0 || l < 0 || k == l) throw Err(CCSD_ERR_ARG, "state indices must differ and be >= 0");
  if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
  if (k > nr || l > nr) throw Err(CCSD_ERR_ARG, "state index beyond the solved roots");
  if ((k > 0 || l > 0) && !(c->have_right && c->have_left)) throw Err(CCSD_ERR_STATE, "EOM states not solved");
}

}  // namespace

extern "C" {

ccsd_status ccsd_transition_density(ccsd_handle c, int k, int l, double* D) {
  return guarded(c, [&] {
    if (!D) throw Err(CCSD_ERR_ARG, "null pointer");
    check_pair(c, k, l);
    ensure_cache(c);
    const int64_t nn = (int64_t)c->n * c->n;
    DevBuf Dt(nn);
    {
      PrecScope fp64(c, refining(c) ? fp64_prec(c) : c->ex->precision());
      transition_density(c, k, l, Dt.p);
    }
    from_device(c, Dt.p, nn, D);
    sync(c);
  });
}

ccsd_status ccsd_connection_term(ccsd_handle c, int k, int l, int ndir, const double* W, double* O) {
  return guarded(c, [&] {
    if (ndir < 1 || !W || !O) throw Err(CCSD_ERR_ARG, "bad arguments");
    check_pair(c, k, l);
    ensure_cache(c);
    const int n = c->n;
    const int64_t nn = (int64_t)n * n;
    DevBuf Dt(nn), Da(nn), out(1), tmp;
    {
      PrecScope fp64(c, refining(c) ? fp64_prec(c) : c->ex->precision());
      transition_density(c, k, l, Dt.p);
    }
    // Da = (D - D^T) / 2, then O[d] = <Da, W[d]>
    launch_antisymmetric_part(n, Dt.p, Da.p, c->st);
    const bool wdev = is_device_ptr(W);
    double* work = c->ex->scratch(1024);
    for (int d = 0; d < ndir; ++d) {
      const double* wp = W + d * nn;
      if (!wdev) {
        to_device(c, wp, nn, tmp);
        wp = tmp.p;
      }
      launch_dot(nn, Da.p, wp, out.p, work, c->st);
      CUDA_OK(cudaMemcpyAsync(O + d, out.p, sizeof(double), cudaMemcpyDefault, c->st));
      sync(c);
    }
  });
}

}  // extern "C"

namespace {
// N_k^L = 1/|<HF|(l0 + L_k) exp(-T)|| (the left state has no component beyond the doubles):
// a_0 = <psi^L|HF> = l0 - <L|(t1, t2 - t1 t1)>, a_mu = <L|tau_mu (1 - T1)|HF>, and the
// biorthonormal-bra metric of a
double left_norm(ccsd_ctx* c, int k) {
  if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
  if (k < 0 || k > (int)c->omega.size()) throw Err(CCSD_ERR_ARG, "state index beyond the solved roots");
  if (k > 0 && !(c->have_right && c->have_left)) throw Err(CCSD_ERR_STATE, "EOM states not solved");
  const int64_t dim = c->dim;
  const double l0 = (k == 0) ? 1.0 : 0.0;
  const double* L = left_vec(c, k);
  DevBuf x(dim), r(dim), a(dim), out(1);
  launch_t2_minus_t1t1(c->vs, c->t.p, x.p, c->st);
  const double a0 = l0 - gram(c, L, dim, 1, x.p, dim, 1)[0];
  // R = (-t1, 0): <L|tau (1 + R)|HF> gives a
  CUDA_OK(cudaMemsetAsync(r.p, 0, dim * sizeof(double), c->st));
  launch_axpby(c->n1, -1.0, c->t.p, 0.0, r.p, c->st);
  launch_tau_expectation(c->vs, 1.0, L, r.p, a.p, c->st);
  launch_bra_metric(c->vs, a.p, out.p, c->ex->scratch(1024), c->st);
  double q = 0.0;
  CUDA_OK(cudaMemcpyAsync(&q, out.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  sync(c);
  const double norm2 = a0 * a0 + q;
  if (!(norm2 > 0.0)) throw Err(CCSD_ERR_NOT_CONVERGED, "left state of zero norm");
  return 1.0 / std::sqrt(norm2);
}

}  // namespace

extern "C" {

ccsd_status ccsd_left_norm(ccsd_handle c, int k, double* N) {
  return guarded(c, [&] {
    if (!N) throw Err(CCSD_ERR_ARG, "null pointer");
    *N = left_norm(c, k);
  });
}

ccsd_status ccsd_normalized_coupling(ccsd_handle c, int k, int l, int ndir, const double* dh, const double* dB,
                                     double* F) {
  return guarded(c, [&] {
    if (ndir < 1 || !dh || !dB || !F) throw Err(CCSD_ERR_ARG, "bad arguments");
    check_pair(c, k, l);
    const double nk = left_norm(c, k), nl = left_norm(c, l);
    std::vector<double> fkl(ndir), flk(ndir);
    compute_densities(c, k, l);
    contract_densities(c, ndir, dh, dB, fkl.data());
    compute_densities(c, l, k);
    contract_densities(c, ndir, dh, dB, flk.data());
    for (int d = 0; d < ndir; ++d) F[d] = 0.5 * (nk / nl * fkl[d] - nl / nk * flk[d]);
  });
}

ccsd_status ccsd_gradient_densities(ccsd_handle c, int k, double* D, double* Z) {
  return guarded(c, [&] {
    if (!D) throw Err(CCSD_ERR_ARG, "null pointer");
    compute_gradient_densities(c, k);
    const int64_t nn = (int64_t)c->n * c->n;
    from_device(c, c->Dd.p, nn, D);
    if (Z) from_device(c, c->Zd.p, (int64_t)c->naux * nn, Z);
    sync(c);
  });
}

ccsd_status ccsd_energy_gradient(ccsd_handle c, int k, int ndir, const double* dh, const double* dB, double* g) {
  return guarded(c, [&] {
    if (ndir < 1 || !dh || !dB || !g) throw Err(CCSD_ERR_ARG, "bad arguments");
    compute_gradient_densities(c, k);
    contract_densities(c, ndir, dh, dB, g);
  });
}

ccsd_status ccsd_branching_plane(ccsd_handle c, int k, int l, int ndir, const double* dh, const double* dB,
                                 double* out) {
  return guarded(c, [&] {
    if (ndir < 1 || !dh || !dB || !out) throw Err(CCSD_ERR_ARG, "bad arguments");
    if (k < 1 || l < 1 || k == l) throw Err(CCSD_ERR_ARG, "branching plane of two distinct excited states");
    std::vector<double> gk(ndir), gl(ndir), f(ndir);
    compute_gradient_densities(c, k);
    contract_densities(c, ndir, dh, dB, gk.data());
    compute_gradient_densities(c, l);
    contract_densities(c, ndir, dh, dB, gl.data());
    compute_densities(c, k, l);
    contract_densities(c, ndir, dh, dB, f.data());
    const double gap = omega_of(c, l) - omega_of(c, k);  // E_l - E_k
    DevBuf d(6 * (int64_t)ndir);
    CUDA_OK(cudaMemcpyAsync(d.p, gk.data(), ndir * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CUDA_OK(cudaMemcpyAsync(d.p + ndir, gl.data(), ndir * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CUDA_OK(cudaMemcpyAsync(d.p + 2 * ndir, f.data(), ndir * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_branching_plane(ndir, gap, d.p, d.p + ndir, d.p + 2 * ndir, d.p + 3 * ndir, c->st);
    from_device(c, d.p + 3 * ndir, 3 * (int64_t)ndir, out);
    sync(c);
  });
}

ccsd_status ccsd_stats(ccsd_handle c, double* flops_fp64, double* flops_tc, long long* gemms, long long* tc_gemms) {
  return guarded(c, [&] {
    if (flops_fp64) *flops_fp64 = c->ex->stats.gemm_flops;
    if (flops_tc) *flops_tc = c->ex->stats.tc_flops;
    if (gemms) *gemms = c->ex->stats.gemm_calls;
    if (tc_gemms) *tc_gemms = c->ex->stats.tc_calls;
  });
}

}  // extern "C"

namespace ccsd {
// Internal accessor for noalloc.cu: the densities of the pair (k, l) if they are
// the ones held by the handle, with the sizes, stream and device.  Allocates nothing.
bool held_densities(ccsd_handle c, int k, int l, const double** D, const double** Z, int* n, int* naux,
                    cudaStream_t* st, int* device) {
  if (!c || c->dens_k != k || c->dens_l != l || !c->Dd.p || !c->Zd.p) return false;
  *D = c->Dd.p;
  *Z = c->Zd.p;
  *n = c->n;
  *naux = c->naux;
  *st = c->st;
  *device = c->device;
  return true;
}
void set_error(ccsd_handle c, const char* msg) {
  if (c) c->err = msg;
}
}  // namespace ccsd

namespace {
// status-returning wrapper for calls without a handle
template <typename F>
ccsd_status unguarded(F&& f) {
  try {
    f();
    return CCSD_OK;
  } catch (const Err& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const OutOfMemory& e) {
    g_last_error = e.what();
    return CCSD_ERR_OOM;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return CCSD_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return g_last_error.find("out of memory") != std::string::npos ? CCSD_ERR_OOM : CCSD_ERR_CUDA;
  }
}

// device copy of a float array given as host or device memory
void floats_to_device(const float* src, int64_t n, DevBuf& dst) {
  dst.alloc((n + 1) / 2);
  CUDA_OK(cudaMemcpy(dst.p, src, n * sizeof(float), cudaMemcpyDefault));
}
}  // namespace

extern "C" {


ccsd_status ccsd_mlp_train(const float* X, const float* T, long long n, int steps, int batch, float lr,
                           unsigned long long seed, float* model_out, float* final_loss) {
  if (!X || !T || !model_out || n < 1 || steps < 0 || batch < 1) return CCSD_ERR_ARG;
  return unguarded([&] {
    // normalisation from the data (host copies)
    std::vector<float> hx(n * 3), ht(n);
    CUDA_OK(cudaMemcpy(hx.data(), X, n * 3 * sizeof(float), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(ht.data(), T, n * sizeof(float), cudaMemcpyDefault));
    std::vector<float> model(mlp::kParams, 0.f);
    mlp::init_weights(model.data(), seed);
    for (int d = 0; d < 3; ++d) {
      double s = 0, s2 = 0;
      for (long long r = 0; r < n; ++r) {
        s += hx[r * 3 + d];
        s2 += (double)hx[r * 3 + d] * hx[r * 3 + d];
      }
      double mean = s / n, var = std::max(s2 / n - mean * mean, 1e-30);
      model[mlp::kTrainable + d] = (float)mean;
      model[mlp::kTrainable + 3 + d] = (float)std::sqrt(var);
    }
    double t2 = 0;
    for (long long r = 0; r < n; ++r) t2 += (double)ht[r] * ht[r];
    model[mlp::kTrainable + 6] = (float)std::max(std::sqrt(t2 / n), 1e-30);
    DevBuf dX, dT, dM, dG((mlp::kTrainable + 1) / 2), dm((mlp::kTrainable + 1) / 2), dv((mlp::kTrainable + 1) / 2),
        didx(batch), dloss(1);
    floats_to_device(hx.data(), n * 3, dX);
    floats_to_device(ht.data(), n, dT);
    floats_to_device(model.data(), mlp::kParams, dM);
    CUDA_OK(cudaMemset(dm.p, 0, mlp::kTrainable * sizeof(float)));
    CUDA_OK(cudaMemset(dv.p, 0, mlp::kTrainable * sizeof(float)));
    const int b = (int)std::min<long long>(batch, n);
    for (int s = 0; s < steps; ++s) {
      const float rate = 0.5f * lr * (1.f + std::cos(3.14159265f * (float)s / (float)std::max(steps, 1)));
      mlp::sample((int64_t*)didx.p, b, n, seed ^ 0x5bd1e995ull, (unsigned long long)s, 0);
      mlp::gradient((const float*)dM.p, (const float*)dX.p, (const float*)dT.p, (const int64_t*)didx.p, b,
                    (float*)dG.p, (float*)dloss.p, 0);
      mlp::adam((float*)dM.p, (const float*)dG.p, (float*)dm.p, (float*)dv.p, rate, s + 1, 0);
    }
    if (final_loss) {
      mlp::gradient((const float*)dM.p, (const float*)dX.p, (const float*)dT.p, nullptr, n, (float*)dG.p,
                    (float*)dloss.p, 0);
      CUDA_OK(cudaMemcpy(final_loss, dloss.p, sizeof(float), cudaMemcpyDeviceToHost));
    }
    CUDA_OK(cudaMemcpy(model_out, dM.p, mlp::kParams * sizeof(float), cudaMemcpyDefault));
    CUDA_OK(cudaDeviceSynchronize());
  });
}

ccsd_status ccsd_mlp_predict(const float* model, const float* X, long long n, float* out) {
  if (!model || !X || !out || n < 1) return CCSD_ERR_ARG;
  return unguarded([&] {
    // device arrays are used in place; host arrays are staged
    DevBuf dM, dX, dO;
    const float* m = model;
    const float* x = X;
    float* o = out;
    if (!is_device_ptr(model)) {
      floats_to_device(model, mlp::kParams, dM);
      m = (const float*)dM.p;
    }
    if (!is_device_ptr(X)) {
      floats_to_device(X, n * 3, dX);
      x = (const float*)dX.p;
    }
    const bool odev = is_device_ptr(out);
    if (!odev) {
      dO.alloc((n + 1) / 2);
      o = (float*)dO.p;
    }
    mlp::predict(m, x, n, o, 0);
    if (!odev) CUDA_OK(cudaMemcpy(out, dO.p, n * sizeof(float), cudaMemcpyDefault));
    CUDA_OK(cudaDeviceSynchronize());
  });
}

ccsd_status ccsd_mlp_gradient(const float* model, const float* X, const float* T, long long n, float* grad,
                              float* loss) {
  if (!model || !X || !T || !grad || n < 1) return CCSD_ERR_ARG;
  return unguarded([&] {
    DevBuf dM, dX, dT, dG((mlp::kTrainable + 1) / 2), dL(1);
    floats_to_device(model, mlp::kParams, dM);
    floats_to_device(X, n * 3, dX);
    floats_to_device(T, n, dT);
    mlp::gradient((const float*)dM.p, (const float*)dX.p, (const float*)dT.p, nullptr, n, (float*)dG.p,
                  (float*)dL.p, 0);
    CUDA_OK(cudaMemcpy(grad, dG.p, mlp::kTrainable * sizeof(float), cudaMemcpyDefault));
    if (loss) CUDA_OK(cudaMemcpy(loss, dL.p, sizeof(float), cudaMemcpyDeviceToHost));
  });
}

ccsd_status ccsd_guess_features(ccsd_handle c, float* X) {
  return guarded(c, [&] {
    if (!X) throw Err(CCSD_ERR_ARG, "null output");
    const int64_t n2 = c->dim - c->n1;
    const double* gov = c->ex->ptr(c->P.cp.g.id("Govov"));
    if (is_device_ptr(X)) {
      mlp::features(gov, c->eps.p, c->o, c->v, X, c->st);
    } else {
      DevBuf dX((n2 * 3 + 1) / 2);
      mlp::features(gov, c->eps.p, c->o, c->v, (float*)dX.p, c->st);
      CUDA_OK(cudaMemcpyAsync(X, dX.p, n2 * 3 * sizeof(float), cudaMemcpyDefault, c->st));
    }
    sync(c);
  });
}

ccsd_status ccsd_set_guess_model(ccsd_handle c, const float* model) {
  return guarded(c, [&] {
    if (!model) {
      c->guess_model.release();
      return;
    }
    floats_to_device(model, mlp::kParams, c->guess_model);
  });
}

ccsd_status ccsd_set_multiplier_guess_model(ccsd_handle c, const float* model) {
  return guarded(c, [&] {
    if (!model) {
      c->mult_model.release();
      return;
    }
    floats_to_device(model, mlp::kParams, c->mult_model);
  });
}

ccsd_status ccsd_guess_targets(ccsd_handle c, int which, float* X, float* T) {
  return guarded(c, [&] {
    if (!X || !T || (which != CCSD_GUESS_AMPLITUDES && which != CCSD_GUESS_MULTIPLIERS))
      throw Err(CCSD_ERR_ARG, "bad arguments");
    if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
    const int64_t n2 = c->dim - c->n1;
    const double* gov = c->ex->ptr(c->P.cp.g.id("Govov"));
    DevBuf dX((n2 * 3 + 1) / 2), dT((n2 + 1) / 2), x0;
    const double* start = nullptr;  // amplitudes: t_MP2 from the integrals
    const double* conv = c->t.p + c->n1;
    if (which == CCSD_GUESS_MULTIPLIERS) {
      x0.alloc(c->dim);
      launch_precond(c->vs, c->eps.p, c->eta.p, x0.p, 0.0, c->st);
      launch_axpby(c->dim, 0.0, x0.p, -1.0, x0.p, c->st);
      start = x0.p + c->n1;
      conv = c->lam.p + c->n1;
    }
    mlp::features(gov, c->eps.p, c->o, c->v, (float*)dX.p, c->st, start);
    mlp::targets(conv, (const float*)dX.p, n2, (float*)dT.p, c->st);
    CUDA_OK(cudaMemcpyAsync(X, dX.p, n2 * 3 * sizeof(float), cudaMemcpyDefault, c->st));
    CUDA_OK(cudaMemcpyAsync(T, dT.p, n2 * sizeof(float), cudaMemcpyDefault, c->st));
    sync(c);
  });
}

ccsd_status ccsd_guess_doubles(ccsd_handle c, int which, const float* model, double* x2) {
  return guarded(c, [&] {
    if (!x2 || (which != CCSD_GUESS_AMPLITUDES && which != CCSD_GUESS_MULTIPLIERS))
      throw Err(CCSD_ERR_ARG, "bad arguments");
    const int64_t n2 = c->dim - c->n1;
    const double* gov = c->ex->ptr(c->P.cp.g.id("Govov"));
    DevBuf start(c->dim), dX((n2 * 3 + 1) / 2);
    if (which == CCSD_GUESS_MULTIPLIERS) {
      if (!c->have_ground) throw Err(CCSD_ERR_STATE, "ground state not solved");
      launch_precond(c->vs, c->eps.p, c->eta.p, start.p, 0.0, c->st);
      launch_axpby(c->dim, 0.0, start.p, -1.0, start.p, c->st);
      mlp::features(gov, c->eps.p, c->o, c->v, (float*)dX.p, c->st, start.p + c->n1);
    } else {
      // the first-order doubles t_MP2 = -(ia|jb)/D (FP64); the features carry them in FP32
      mlp::features(gov, c->eps.p, c->o, c->v, (float*)dX.p, c->st);
      mlp::mp2_doubles(gov, c->eps.p, c->o, c->v, start.p + c->n1, c->st);
    }
    if (model) {
      DevBuf m, delta((n2 + 1) / 2);
      floats_to_device(model, mlp::kParams, m);
      mlp::predict((const float*)m.p, (const float*)dX.p, n2, (float*)delta.p, c->st);
      mlp::add_delta(start.p + c->n1, (const float*)delta.p, n2, c->st);
    }
    from_device(c, start.p + c->n1, n2, x2);
    sync(c);
  });
}

ccsd_status ccsd_solve_iterations(ccsd_handle c, int* ground, int* lambda, int* zeta) {
  return guarded(c, [&] {
    if (ground) *ground = c->iters_ground;
    if (lambda) *lambda = c->iters_lambda;
    if (zeta) *zeta = c->iters_zeta;
  });
}

ccsd_status ccsd_set_wait_budget(ccsd_handle c, long long cycles) {
  return guarded(c, [&] {
    if (cycles < 0) throw Err(CCSD_ERR_ARG, "wait budget must be >= 0");
    c->ex->wait_cycles = cycles;
    if (c->hx) c->hx->wait_cycles = cycles;
  });
}

ccsd_status ccsd_inject_stall(ccsd_handle c) {
  return guarded(c, [&] {
    if (c->opt.precision != CCSD_PREC_MIXED) throw Err(CCSD_ERR_STATE, "stall injection needs a mixed-precision handle");
    c->ex->stall_next = true;
  });
}

ccsd_status ccsd_profile_start(ccsd_handle c) {
  return guarded(c, [&] {
    c->ex->collect();
    c->ex->profile(true);
    c->prof_launch0 = kernel_launches();
  });
}

ccsd_status ccsd_profile_stop(ccsd_handle c, ccsd_profile_data* out) {
  return guarded(c, [&] {
    Executor::ProfTotals t = c->ex->collect();
    c->ex->profile(false);
    if (out) {
      out->launches = kernel_launches() - c->prof_launch0;
      out->tc_launches = t.tc_launches;
      out->tc_ms = t.tc_ms;
      out->tc_flops = t.tc_flops;
      out->tc_issued_flops = t.tc_issued;
      out->fp64_launches = t.fp64_launches;
      out->fp64_ms = t.fp64_ms;
      out->fp64_flops = t.fp64_flops;
      out->top_launches = t.top_launches;
      out->top_ms = t.top_ms;
      out->top_flops = t.top_flops;
      out->top_issued_flops = t.top_issued;
      out->ladder_launches = t.ladder_launches;
      out->ladder_ms = t.ladder_ms;
      out->ladder_flops = t.ladder_flops;
      out->ladder_issued_flops = t.ladder_issued;
    }
  });
}

ccsd_status ccsd_profile_records(ccsd_handle c, ccsd_profile_record* out, int max, int* count) {
  return guarded(c, [&] {
    if (!count || max < 0 || (max > 0 && !out)) throw Err(CCSD_ERR_ARG, "profile records: count, max or out");
    const auto& lines = c->ex->profile_lines();
    *count = (int)lines.size();
    const int n = std::min<int>(max, (int)lines.size());
    for (int i = 0; i < n; ++i) {
      const auto& l = lines[i];
      ccsd_profile_record& r = out[i];
      std::memset(&r, 0, sizeof(r));
      std::snprintf(r.label, sizeof(r.label), "%s", l.label.c_str());
      r.engine = l.engine;
      r.ladder = l.ladder ? 1 : 0;
      r.batch = l.batch;
      r.m = l.m;
      r.n = l.n;
      r.k = l.k;
      r.ms = l.ms;
      r.flops = l.flops;
      r.issued_flops = l.issued;
    }
  });
}

long long ccsd_describe_program(const char* which, char* buf, size_t len) {
  try {
    Programs P;
    build_programs(P);
    const Prog* p = nullptr;
    std::string w = which ? which : "";
    if (w == "fwd") p = &P.cp.fwd;
    else if (w == "jvp") p = &P.jvp_z;
    else if (w == "vjp") p = &P.vjp_z;
    else if (w == "hvp") p = &P.hvp;
    else if (w == "dens1") p = &P.dens1;
    else if (w == "dens0") p = &P.dens0;
    HFPrograms H;
    const Graph* g = &P.cp.g;
    if (!p && w.rfind("hf_", 0) == 0) {
      build_hf_programs(H);
      g = &H.g;
      if (w == "hf_fock") p = &H.fock;
      else if (w == "hf_A") p = &H.hfA;
      else if (w == "hf_rotT") p = &H.rotT;
      else if (w == "hf_kdens") p = &H.kdens;
      else if (w == "hf_rotate") p = &H.rotate;
    }
    if (!p) return -1;
    std::string s = dump(*g, *p);
    if (buf && len > 0) {
      size_t m = std::min(len - 1, s.size());
      std::memcpy(buf, s.data(), m);
      buf[m] = 0;
    }
    return (long long)s.size();
  } catch (...) {
    return -1;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches of systems: block transforms of all systems as one CUDA graph launch
// ---------------------------------------------------------------------------
struct ccsd_batch_ctx {
  std::vector<ccsd_ctx*> sys;
  std::vector<cudaStream_t> orig, own;  // each handle's stream before the batch, and the batch's streams
  cudaStream_t cap = nullptr;           // capture / launch stream
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  int nvec = 8;
  std::vector<std::unique_ptr<DevBuf>> X, Y, W, G;  // per system [nvec][dim] staging
  struct Graph {
    int side;
    std::vector<char> mask;
    cudaGraphExec_t exec;
    long long nodes;
    std::vector<uint64_t> epochs;  // the systems' operand-cache epochs at capture
  };
  std::vector<Graph> graphs;
  long long launches = 0, captures = 0, last_nodes = 0;
  std::string err;
};

namespace {

template <typename F>
ccsd_status batch_guarded(ccsd_batch_ctx* b, F&& f) {
  if (!b) return CCSD_ERR_ARG;
  try {
    f();
    return CCSD_OK;
  } catch (const Err& e) {
    b->err = e.what();
    return e.code;
  } catch (const DeviceTimeout& e) {
    b->err = e.what();
    return CCSD_ERR_TIMEOUT;
  } catch (const OutOfMemory& e) {
    b->err = e.what();
    return CCSD_ERR_OOM;
  } catch (const std::bad_alloc&) {
    b->err = "host allocation failed";
    return CCSD_ERR_OOM;
  } catch (const std::exception& e) {
    b->err = e.what();
    return b->err.find("out of memory") != std::string::npos ? CCSD_ERR_OOM : CCSD_ERR_CUDA;
  }
}

// f(i) for i < n on up to hardware_concurrency host threads (each system's host-side
// solver work runs on its own stream, so systems proceed independently); the first
// exception is rethrown after all threads have joined
template <typename F>
void parallel_for(int n, F&& f) {
  int dev = 0;
  CUDA_OK(cudaGetDevice(&dev));
  const int nt = std::max(1, std::min<int>(n, (int)std::max(1u, std::thread::hardware_concurrency())));
  std::atomic<int> next{0};
  std::vector<std::exception_ptr> err(n);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&] {
      cudaSetDevice(dev);
      for (;;) {
        const int i = next++;
        if (i >= n) break;
        try {
          f(i);
        } catch (...) {
          err[i] = std::current_exception();
        }
      }
    });
  for (auto& t : th) t.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}

// system s's block transform of its staging vectors, on its own stream, without synchronising
void batch_block(ccsd_batch_ctx* b, int s, int side) {
  ccsd_ctx* c = b->sys[s];
  if (side == 0) {
    Executor& ex = *c->ex;
    auto& P = c->P;
    ex.set_nvec(b->nvec);
    ex.bind(P.zR1, b->X[s]->p, c->dim);
    ex.bind(P.zR2, b->X[s]->p + c->n1, c->dim);
    ex.bind(P.zAR1, b->Y[s]->p, c->dim);
    ex.bind(P.zAR2, b->Y[s]->p + c->n1, c->dim);
    ex.bind(P.zAE, c->gsc.p);
    ex.run(P.jvp_z);
  } else {
    left_block_into(c, b->X[s]->p, b->Y[s]->p, b->nvec, b->W[s]->p, b->G[s]->p);
  }
}

// Y_s = transform of X_s for the systems in mask: one graph launch once captured
void batch_run(ccsd_batch_ctx* b, int side, const std::vector<char>& mask) {
  const int ns = (int)b->sys.size();
  for (int s = 0; s < ns; ++s)
    if (mask[s]) {
      ensure_cache(b->sys[s]);
      if (side == 1 && !b->W[s]) {
        b->W[s].reset(new DevBuf(b->nvec * b->sys[s]->dim));
        b->G[s].reset(new DevBuf(b->nvec * b->sys[s]->dim));
      }
    }
  std::vector<uint64_t> epochs(ns);
  for (int s = 0; s < ns; ++s) epochs[s] = b->sys[s]->ex->cache_epoch();
  // graphs whose captured operand slices were dropped since (new amplitudes) are stale
  for (size_t i = 0; i < b->graphs.size();) {
    if (b->graphs[i].epochs != epochs) {
      cudaGraphExecDestroy(b->graphs[i].exec);
      b->graphs.erase(b->graphs.begin() + i);
    } else {
      ++i;
    }
  }
  for (auto& g : b->graphs)
    if (g.side == side && g.mask == mask) {
      CUDA_OK(cudaGraphLaunch(g.exec, b->cap));
      CUDA_OK(cudaStreamSynchronize(b->cap));
      ++b->launches;
      count_launches(g.nodes);
      for (int s = 0; s < ns; ++s)
        if (mask[s] && b->sys[s]->ex->tc_error() != 0)
          throw DeviceTimeout("a tensor-core kernel wait exceeded its budget");
      return;
    }
  // first use of this (side, mask): run directly (the result is this call's), then capture
  for (int s = 0; s < ns; ++s)
    if (mask[s]) batch_block(b, s, side);
  for (int s = 0; s < ns; ++s)
    if (mask[s]) {
      CUDA_OK(cudaStreamSynchronize(b->sys[s]->st));
      if (b->sys[s]->ex->tc_error() != 0) throw DeviceTimeout("a tensor-core kernel wait exceeded its budget");
    }
  cudaGraph_t graph = nullptr;
  CUDA_OK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  try {
    CUDA_OK(cudaEventRecord(b->fork, b->cap));
    for (int s = 0; s < ns; ++s) {
      if (!mask[s]) continue;
      ccsd_ctx* c = b->sys[s];
      CUDA_OK(cudaStreamWaitEvent(c->st, b->fork, 0));
      c->ex->capturing = true;
      batch_block(b, s, side);
      c->ex->capturing = false;
      CUDA_OK(cudaEventRecord(b->join[s], c->st));
      CUDA_OK(cudaStreamWaitEvent(b->cap, b->join[s], 0));
    }
    CUDA_OK(cudaStreamEndCapture(b->cap, &graph));
  } catch (...) {
    for (ccsd_ctx* c : b->sys) c->ex->capturing = false;
    cudaGraph_t g2 = nullptr;
    cudaStreamEndCapture(b->cap, &g2);
    if (g2) cudaGraphDestroy(g2);
    cudaGetLastError();
    throw;
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  size_t nnodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nnodes);
  cudaGraphDestroy(graph);
  CUDA_OK(e);
  ++b->captures;
  b->last_nodes = (long long)nnodes;
  for (int s = 0; s < ns; ++s) epochs[s] = b->sys[s]->ex->cache_epoch();
  b->graphs.push_back({side, mask, exec, (long long)nnodes, epochs});
}

void batch_release(ccsd_batch_ctx* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
  for (size_t s = 0; s < b->sys.size(); ++s) {
    ccsd_ctx* c = b->sys[s];
    cudaStreamSynchronize(c->st);
    c->st = b->orig[s];
    c->ex->set_stream(b->orig[s]);
  }
  for (cudaStream_t st : b->own) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  b->own.clear();
  b->join.clear();
  b->fork = nullptr;
  b->cap = nullptr;
}

}  // namespace

extern "C" {

ccsd_status ccsd_batch_create(int nsys, const ccsd_handle* systems, int nvec, ccsd_batch* out) {
  if (!out) return CCSD_ERR_ARG;
  *out = nullptr;
  if (nsys < 1 || !systems || nvec < 1 || nvec > 16) return CCSD_ERR_ARG;
  for (int s = 0; s < nsys; ++s) {
    // a batch captures its systems' work into CUDA graphs, whose temporaries are graph
    // memory nodes: systems with allocator callbacks cannot take part
    if (!systems[s] || systems[s]->allocator.custom()) return CCSD_ERR_ARG;
    for (int r = 0; r < s; ++r)
      if (systems[r] == systems[s]) return CCSD_ERR_ARG;
  }
  std::unique_ptr<ccsd_batch_ctx> b(new ccsd_batch_ctx);
  b->nvec = nvec;
  ccsd_status st = batch_guarded(b.get(), [&] {
    CUDA_OK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    CUDA_OK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (int s = 0; s < nsys; ++s) {
      ccsd_ctx* c = systems[s];
      cudaStream_t st = nullptr;
      CUDA_OK(cudaStreamSynchronize(c->st));
      CUDA_OK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      cudaEvent_t e = nullptr;
      CUDA_OK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      b->own.push_back(st);
      b->join.push_back(e);
      b->orig.push_back(c->st);
      b->sys.push_back(c);
      c->st = st;
      c->ex->set_stream(st);
      b->X.emplace_back(new DevBuf(nvec * c->dim));
      b->Y.emplace_back(new DevBuf(nvec * c->dim));
      CUDA_OK(cudaMemsetAsync(b->X.back()->p, 0, nvec * c->dim * sizeof(double), st));
      b->W.emplace_back(nullptr);
      b->G.emplace_back(nullptr);
    }
  });
  if (st != CCSD_OK) {
    batch_release(b.get());
    return st;
  }
  *out = b.release();
  return CCSD_OK;
}

ccsd_status ccsd_batch_transform(ccsd_batch b, int side, const double* const* x, double* const* y) {
  return batch_guarded(b, [&] {
    if ((side != 0 && side != 1) || !x || !y) throw Err(CCSD_ERR_ARG, "bad arguments");
    const int ns = (int)b->sys.size();
    for (int s = 0; s < ns; ++s) {
      if (!x[s] || !y[s]) throw Err(CCSD_ERR_ARG, "null vector array");
      if (!b->sys[s]->have_ground) throw Err(CCSD_ERR_STATE, "a system has no amplitudes");
    }
    for (int s = 0; s < ns; ++s) {
      ccsd_ctx* c = b->sys[s];
      CUDA_OK(cudaMemcpyAsync(b->X[s]->p, x[s], b->nvec * c->dim * sizeof(double), cudaMemcpyDefault, c->st));
      CUDA_OK(cudaStreamSynchronize(c->st));
    }
    batch_run(b, side, std::vector<char>(ns, 1));
    for (int s = 0; s < ns; ++s) {
      ccsd_ctx* c = b->sys[s];
      CUDA_OK(cudaMemcpyAsync(y[s], b->Y[s]->p, b->nvec * c->dim * sizeof(double), cudaMemcpyDefault, c->st));
    }
    for (int s = 0; s < ns; ++s) CUDA_OK(cudaStreamSynchronize(b->sys[s]->st));
  });
}

ccsd_status ccsd_batch_eom_solve(ccsd_batch b, int side, int nroots, double* omega, int* iters) {
  return batch_guarded(b, [&] {
    const int ns = (int)b->sys.size();
    if ((side != 0 && side != 1) || nroots < 1 || nroots > b->nvec) throw Err(CCSD_ERR_ARG, "bad arguments");
    for (ccsd_ctx* c : b->sys) {
      if (nroots > c->n1) throw Err(CCSD_ERR_ARG, "nroots exceeds a system's singles dimension");
      if (!c->have_ground) throw Err(CCSD_ERR_STATE, "a system has no ground state");
      if (side == 1 && (!c->have_right || (int)c->omega.size() != nroots))
        throw Err(CCSD_ERR_STATE, "side 1 needs the right solve with the same nroots first");
    }
    std::vector<std::unique_ptr<Davidson>> d(ns);
    parallel_for(ns, [&](int s) {
      ccsd_ctx* c = b->sys[s];
      const double tol = refining(c) ? std::max(c->opt.tol_eom, 10.0 * c->opt.tol_switch) : c->opt.tol_eom;
      d[s].reset(new Davidson(c, side, nroots, tol, side == 1 ? &c->R : nullptr));
      if (side == 1) d[s]->targets = c->omega;
    });
    std::vector<char> done(ns, 0), mask(ns, 1);
    std::vector<int> it(ns, 0);
    int left = ns;
    while (left > 0) {
      // transform every pending vector, nvec per system and launch
      std::vector<int> off(ns, 0);
      for (;;) {
        bool any = false;
        std::vector<int> k(ns, 0);
        for (int s = 0; s < ns; ++s) {
          if (!mask[s]) continue;
          ccsd_ctx* c = b->sys[s];
          if (!done[s]) k[s] = std::max(0, std::min(b->nvec, d[s]->count - off[s]));
          if (k[s] > 0) {
            any = true;
            CUDA_OK(cudaMemcpyAsync(b->X[s]->p, d[s]->vin(off[s]), k[s] * c->dim * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->st));
          }
          if (k[s] < b->nvec)
            CUDA_OK(cudaMemsetAsync(b->X[s]->p + k[s] * c->dim, 0, (b->nvec - k[s]) * c->dim * sizeof(double),
                                    c->st));
          CUDA_OK(cudaStreamSynchronize(c->st));
        }
        if (!any) break;
        batch_run(b, side, mask);
        for (int s = 0; s < ns; ++s)
          if (k[s] > 0) {
            ccsd_ctx* c = b->sys[s];
            CUDA_OK(cudaMemcpyAsync(d[s]->vout(off[s]), b->Y[s]->p, k[s] * c->dim * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->st));
            off[s] += k[s];
          }
      }
      std::vector<char> conv(ns, 0);
      parallel_for(ns, [&](int s) {
        if (done[s]) return;
        CUDA_OK(cudaStreamSynchronize(b->sys[s]->st));
        conv[s] = d[s]->advance() ? 1 : 0;
      });
      for (int s = 0; s < ns; ++s)
        if (!done[s] && conv[s]) {
          done[s] = 1;
          --left;
        }
      // drop converged systems from the launched set once a quarter of it is idle
      int active = 0, idle = 0;
      for (int s = 0; s < ns; ++s)
        if (mask[s]) (done[s] ? idle : active)++;
      if (active > 0 && 4 * idle >= active + idle)
        for (int s = 0; s < ns; ++s)
          if (done[s]) mask[s] = 0;
    }
    parallel_for(ns, [&](int s) {
      ccsd_ctx* c = b->sys[s];
      std::vector<double> w = d[s]->omega;
      int its = d[s]->iterations;
      std::vector<std::unique_ptr<DevBuf>> vecs;
      d[s]->results(vecs);
      d[s].reset();
      if (refining(c)) its += refine_roots(c, side, w, vecs);  // FP64 refinement of this system alone
      if (side == 0) {
        c->R.swap(vecs);
        finish_right(c, w);
      } else {
        finish_left(c, w, vecs);
      }
      if (omega) std::copy(w.begin(), w.end(), omega + (size_t)s * nroots);
      if (iters) iters[s] = its;
    });
  });
}

ccsd_status ccsd_batch_stats(ccsd_batch b, long long* launches, long long* captures, long long* nodes) {
  if (!b) return CCSD_ERR_ARG;
  if (launches) *launches = b->launches;
  if (captures) *captures = b->captures;
  if (nodes) *nodes = b->last_nodes;
  return CCSD_OK;
}

const char* ccsd_batch_last_error(ccsd_batch b) { return b ? b->err.c_str() : "null batch"; }

void ccsd_batch_destroy(ccsd_batch b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Hartree-Fock orbitals for the relaxed mode
// ---------------------------------------------------------------------------
namespace {

// exp(K) of an antisymmetric n x n matrix (host, row-major) into U (device):
// scaling and squaring with a degree-16 Taylor polynomial (||K / 2^s||_1 <= 1/4,
// truncation error below 1e-20 before squaring); the products run in the FP64 GEMM.
void expm_device(const std::vector<double>& K, int n, double* U, cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  double nrm = 0.0;
  for (int q = 0; q < n; ++q) {
    double col = 0.0;
    for (int p = 0; p < n; ++p) col += std::fabs(K[(int64_t)p * n + q]);
    nrm = std::max(nrm, col);
  }
  int s = 0;
  while (std::ldexp(nrm, -s) > 0.25) ++s;
  std::vector<double> Ks(nn), I(nn, 0.0);
  for (int64_t e = 0; e < nn; ++e) Ks[e] = std::ldexp(K[e], -s);
  for (int p = 0; p < n; ++p) I[(int64_t)p * n + p] = 1.0;
  DevBuf X(nn), T(nn), T2(nn), S(nn);
  CUDA_OK(cudaMemcpyAsync(X.p, Ks.data(), nn * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemcpyAsync(T.p, I.data(), nn * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_OK(cudaMemcpyAsync(S.p, I.data(), nn * sizeof(double), cudaMemcpyHostToDevice, st));
  // C[m][q] = alpha sum_k A[m][k] Y[k][q]: the GEMM's second operand is read as [q][k]
  auto mul = [&](const double* A, const double* Y, double* C, double alpha) {
    GemmArgs g{};
    g.batch = 1;
    g.M = g.N = g.K = n;
    g.A = A;
    g.sAm = n;
    g.sAk = 1;
    g.B = Y;
    g.sBn = 1;
    g.sBk = n;
    g.C = C;
    g.sCm = n;
    g.sCn = 1;
    g.alpha = alpha;
    g.beta = 0.0;
    launch_dgemm(g, st);
  };
  for (int k = 1; k <= 16; ++k) {  // S = sum_k (K/2^s)^k / k!
    mul(T.p, X.p, T2.p, 1.0 / k);
    std::swap(T.p, T2.p);
    launch_axpby(nn, 1.0, T.p, 1.0, S.p, st);
  }
  for (int q = 0; q < s; ++q) {
    mul(S.p, S.p, T2.p, 1.0);
    std::swap(S.p, T2.p);
  }
  CUDA_OK(cudaMemcpyAsync(U, S.p, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_OK(cudaStreamSynchronize(st));
}

}  // namespace

extern "C" {

ccsd_status ccsd_gemm(int form, int splits, int M, int N, int K, double alpha, const double* A, const double* B,
                      double beta, double* C, int reps, double* ms) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || reps < 1) return CCSD_ERR_ARG;
  if (form != CCSD_GEMM_FP64 && form != CCSD_GEMM_SPLIT && form != CCSD_GEMM_FP64_TC) return CCSD_ERR_ARG;
  if (form != CCSD_GEMM_FP64 && beta != 0.0 && beta != 1.0) return CCSD_ERR_ARG;
  if (form == CCSD_GEMM_SPLIT && splits != 2 && splits != 3) return CCSD_ERR_ARG;
  return unguarded([&] {
    const int64_t mk = (int64_t)M * K, nk = (int64_t)N * K, mn = (int64_t)M * N;
    DevBuf dA(mk), dB(nk), dC(mn), dC0(mn);
    CUDA_OK(cudaMemcpy(dA.p, A, mk * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(dB.p, B, nk * sizeof(double), cudaMemcpyDefault));
    if (beta != 0.0)
      CUDA_OK(cudaMemcpy(dC0.p, C, mn * sizeof(double), cudaMemcpyDefault));
    else
      CUDA_OK(cudaMemset(dC0.p, 0, mn * sizeof(double)));
    static const Graph empty;
    cudaStream_t st = nullptr;
    Executor ex(empty, 1, 1, 1, 1, st);
    ex.tc_min_flops = 0.0;
    ex.set_precision(form == CCSD_GEMM_SPLIT ? PREC_MIXED : (form == CCSD_GEMM_FP64_TC ? PREC_FP64_TC : PREC_FP64),
                     form == CCSD_GEMM_SPLIT ? splits : 3);
    Strided ga, gb;
    ga.ndim = gb.ndim = 2;
    ga.ext[0] = M;
    gb.ext[0] = N;
    ga.ext[1] = gb.ext[1] = K;
    ga.s1[0] = gb.s1[0] = K;
    ga.s1[1] = gb.s1[1] = 1;
    ga.s0[0] = ga.s0[1] = gb.s0[0] = gb.s0[1] = 0;
    cudaEvent_t e0, e1;
    CUDA_OK(cudaEventCreate(&e0));
    CUDA_OK(cudaEventCreate(&e1));
    double total = 0.0;
    for (int r = 0; r < reps; ++r) {
      CUDA_OK(cudaMemcpyAsync(dC.p, dC0.p, mn * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CUDA_OK(cudaEventRecord(e0, st));
      if (form == CCSD_GEMM_FP64) {
        GemmArgs g;
        g.batch = 1;
        g.M = M;
        g.N = N;
        g.K = K;
        g.A = dA.p;
        g.sAb = 0;
        g.sAm = K;
        g.sAk = 1;
        g.B = dB.p;
        g.sBb = 0;
        g.sBn = K;
        g.sBk = 1;
        g.C = dC.p;
        g.sCb = 0;
        g.sCm = N;
        g.sCn = 1;
        g.alpha = alpha;
        g.beta = beta;
        launch_dgemm(g, st);
      } else if (!ex.tc_contract(M, N, K, dA.p, ga, dB.p, gb, dC.p, N, 1, alpha, beta, false, false)) {
        throw Err(CCSD_ERR_ARG, "contraction shape not supported by the tensor-core path");
      }
      CUDA_OK(cudaEventRecord(e1, st));
      CUDA_OK(cudaEventSynchronize(e1));
      float t = 0.f;
      CUDA_OK(cudaEventElapsedTime(&t, e0, e1));
      total += t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ex.tc_error()) throw Err(CCSD_ERR_TIMEOUT, "a tensor-core kernel wait timed out");
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaMemcpy(C, dC.p, mn * sizeof(double), cudaMemcpyDefault));
    if (ms) *ms = total / reps;
  });
}

ccsd_status ccsd_scf(const double* eps, const double* h, const double* B, int o, int v, int naux, double tol,
                     double* U_out, double* h_out, double* B_out, int* iters) {
  if (!eps || !h || !B || !U_out || o < 1 || v < 1 || naux < 1 || !(tol > 0.0)) return CCSD_ERR_ARG;
  return unguarded([&] {
    const int n = o + v;
    const int64_t nn = (int64_t)n * n, nz = (int64_t)naux * nn, m = (int64_t)o * v;
    cudaStream_t st = nullptr;
    DevBuf h0(nn), B0(nz), hr(nn), Br(nz), Ud(nn), f(m), ones(o);
    CUDA_OK(cudaMemcpy(h0.p, h, nn * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(B0.p, B, nz * sizeof(double), cudaMemcpyDefault));
    std::vector<double> e(n), one(o, 1.0);
    CUDA_OK(cudaMemcpy(e.data(), eps, n * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(ones.p, one.data(), o * sizeof(double), cudaMemcpyHostToDevice));
    HFPrograms P;
    build_hf_programs(P);
    Executor hx(P.g, o, v, naux, 1, st);
    hx.set_precision(CCSD_PREC_FP64, 3);
    hx.bind(P.ones_o, ones.p);
    hx.bind(P.U, Ud.p);
    hx.bind(P.hr, hr.p);
    hx.bind(P.Br, Br.p);
    hx.bind(P.F, f.p);
    // Newton-type iterations on kappa: F'(exp(K(kappa)))_ia = 0, each step solving
    // J(h', B') dkappa = -F' (J the local derivative dF'/dkappa, not symmetric away from
    // the solution) at the current rotated integrals by GMRES
    std::vector<double> kappa(m, 0.0), fh(m), K(nn);
    int it = 0;
    for (;; ++it) {
      if (it > 100) throw Err(CCSD_ERR_NOT_CONVERGED, "Hartree-Fock equations not converged");
      std::fill(K.begin(), K.end(), 0.0);
      for (int i = 0; i < o; ++i)
        for (int a = 0; a < v; ++a) {
          K[(int64_t)(o + a) * n + i] = kappa[i * v + a];
          K[(int64_t)i * n + o + a] = -kappa[i * v + a];
        }
      expm_device(K, n, Ud.p, st);
      hx.bind(P.h, h0.p);
      hx.bind(P.B, B0.p);
      hx.run(P.rotate);
      hx.bind(P.h, hr.p);
      hx.bind(P.B, Br.p);
      hx.bind(P.F, f.p);
      hx.run(P.fock);
      CUDA_OK(cudaMemcpy(fh.data(), f.p, m * sizeof(double), cudaMemcpyDeviceToHost));
      double fmax = 0.0;
      for (double x : fh) fmax = std::max(fmax, std::fabs(x));
      if (!std::isfinite(fmax)) throw Err(CCSD_ERR_NOT_CONVERGED, "Hartree-Fock iterations diverged");
      if (fmax < tol) break;
      std::vector<double> rhs(m);
      for (int64_t q = 0; q < m; ++q) rhs[q] = -fh[q];
      std::vector<double> dk = hf_solve_general(hx, P, o, v, st, rhs, e, 1e-4, 300);
      for (int64_t q = 0; q < m; ++q) kappa[q] += dk[q];
    }
    CUDA_OK(cudaMemcpy(U_out, Ud.p, nn * sizeof(double), cudaMemcpyDefault));
    if (h_out) CUDA_OK(cudaMemcpy(h_out, hr.p, nn * sizeof(double), cudaMemcpyDefault));
    if (B_out) CUDA_OK(cudaMemcpy(B_out, Br.p, nz * sizeof(double), cudaMemcpyDefault));
    if (iters) *iters = it;
  });
}

ccsd_status ccsd_rotate_integrals(const double* U, const double* h, const double* B, int o, int v, int naux,
                                  double* h_out, double* B_out) {
  if (!U || !h || !B || !h_out || !B_out || o < 1 || v < 1 || naux < 1) return CCSD_ERR_ARG;
  return unguarded([&] {
    const int n = o + v;
    const int64_t nn = (int64_t)n * n, nz = (int64_t)naux * nn;
    DevBuf Ud(nn), hd(nn), Bd(nz), hr(nn), Br(nz);
    CUDA_OK(cudaMemcpy(Ud.p, U, nn * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(hd.p, h, nn * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(Bd.p, B, nz * sizeof(double), cudaMemcpyDefault));
    HFPrograms P;
    build_hf_programs(P);
    Executor hx(P.g, o, v, naux, 1, nullptr);
    hx.set_precision(CCSD_PREC_FP64, 3);
    hx.bind(P.h, hd.p);
    hx.bind(P.B, Bd.p);
    hx.bind(P.U, Ud.p);
    hx.bind(P.hr, hr.p);
    hx.bind(P.Br, Br.p);
    hx.run(P.rotate);
    CUDA_OK(cudaMemcpy(h_out, hr.p, nn * sizeof(double), cudaMemcpyDefault));
    CUDA_OK(cudaMemcpy(B_out, Br.p, nz * sizeof(double), cudaMemcpyDefault));
  });
}

ccsd_status ccsd_get_orbital_multipliers(ccsd_handle c, int k, int l, double* kbar) {
  return guarded(c, [&] {
    if (!c->opt.relax_orbitals) throw Err(CCSD_ERR_STATE, "the handle does not relax orbitals");
    if (!kbar) throw Err(CCSD_ERR_ARG, "null output");
    compute_densities(c, k, l);
    CUDA_OK(cudaMemcpy(kbar, c->kbar.data(), c->kbar.size() * sizeof(double), cudaMemcpyDefault));
  });
}

}  // extern "C"
