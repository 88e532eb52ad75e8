/*
 * ccsd.h -- C ABI of the GB300 library for biorthonormal CCSD derivative
 * couplings (Kjonstad & Koch, "Non-adiabatic derivative coupling elements for
 * the coupled cluster singles and doubles model").
 *
 * Problem statement (Theory section): a closed-shell Hamiltonian with
 * one-electron integrals h_pq and two-electron integrals in Cholesky form
 * g_pqrs = sum_J B^J_pq B^J_rs; the CCSD ground state, EOM-CCSD left/right
 * states, and the biorthonormal derivative coupling F_kl = <psi_k^L | d/dx psi_l^R>
 * (Eq. nac) along a perturbation x of (h, B), evaluated with the Lagrangian of
 * the Lagrangian section (Eqs. for gamma, t-eta, amplituderelax, NAC_NC).
 *
 * Conventions shared by all calls
 * - Orbitals: n = o + v, occupied first.  Arrays are FP64, row-major (C order).
 * - eps[n]: orbital energies; used only for the denominators of the
 *   preconditioners (D_ai = eps_a - eps_i, D_aibj = eps_a + eps_b - eps_i - eps_j).
 * - h[n*n] symmetric; B[naux*n*n] with B^J symmetric in pq.
 * - Amplitude-like vectors have dim = o*v + o*o*v*v entries: singles x[i][a]
 *   followed by doubles x[i][j][a][b] with x_ijab = x_jiba.  The doubles entry is
 *   the packed coefficient of the excitation tau_aibj (ai >= bj) of the
 *   biorthonormal basis, stored at both (i,j,a,b) and (j,i,b,a); inner products
 *   are the packed ones, sum_ai x_ai y_ai + sum_{ai >= bj} x_aibj y_aibj.
 * - Pointers: every array argument may be host or device memory; the library
 *   detects which (cudaPointerGetAttributes) and writes outputs to the same
 *   memory space as given.  The caller owns all buffers it passes.
 * - Streams: all GPU work runs on options.stream (0 = the legacy default
 *   stream).  Calls that return host values synchronise that stream.
 * - Errors: every call returns a ccsd_status; no C++ exception crosses the
 *   ABI.  ccsd_last_error(handle) gives the message of the last failure;
 *   ccsd_last_error(NULL) that of the calling thread's last failed call made
 *   without a handle (ccsd_scf, ccsd_mlp_*, ...).
 * - Threads: a handle must not be used by two threads at once.
 * - State indices: k, l in {0 = ground state, 1..nroots}; the excited states
 *   are those of the last eom_solve_right/left pair.  For k = 0 the left
 *   ground state is <HF|(1 + Lambda) exp(-T).
 */
#ifndef CCSD_GB300_H
#define CCSD_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccsd_ctx* ccsd_handle;

typedef enum {
  CCSD_OK = 0,
  CCSD_ERR_ARG = 1,           /* invalid argument (sizes, NULL, asymmetric B, bad state index) */
  CCSD_ERR_OOM = 2,           /* device allocation failed */
  CCSD_ERR_CUDA = 3,          /* CUDA runtime error */
  CCSD_ERR_STATE = 4,         /* call made before its prerequisites (e.g. EOM before ground) */
  CCSD_ERR_NOT_CONVERGED = 5, /* iteration limit reached */
  CCSD_ERR_COMPLEX_ROOT = 6,  /* a wanted EOM root came out complex (defective intersection) */
  CCSD_ERR_DEGENERATE = 7,    /* omega_l - omega_k below the degeneracy threshold */
  CCSD_ERR_NOT_HF = 8,        /* relax_orbitals = 1 without Hartree-Fock orbitals (F_ia != 0) */
  CCSD_ERR_TIMEOUT = 9        /* a device-side wait exceeded its budget */
} ccsd_status;

/* CCSD_PREC_FP64: every contraction in FP64 (DFMA).
 * CCSD_PREC_MIXED: contractions above tc_min_flops as split-bf16 tensor-core products (FP32
 *   accumulation), optionally refined to the FP64 tolerances (refine, fp64_tc).
 * CCSD_PREC_FP64_TC: contractions above tc_min_flops as FP64-grade tensor-core products (see
 *   fp64_tc below); the solvers run directly to the FP64 tolerances, without refinement. */
enum { CCSD_PREC_FP64 = 0, CCSD_PREC_MIXED = 1, CCSD_PREC_FP64_TC = 2 };
enum { CCSD_GUESS_MP2 = 0 };

typedef struct {
  int precision;        /* CCSD_PREC_FP64, CCSD_PREC_MIXED or CCSD_PREC_FP64_TC; anything else: CCSD_ERR_ARG */
  int splits;           /* mixed mode: bf16 slices per FP64 operand (2 or 3) */
  int relax_orbitals;   /* 0: orbitals fixed and x-independent (unrelaxed coupling); 1: Hartree-Fock
                           orbitals that follow x (Eq. orbitalrelax): the inputs must be Hartree-Fock
                           orbitals (ccsd_scf), else ccsd_create returns CCSD_ERR_NOT_HF */
  double tol_res;       /* ground state: max |Omega| */
  double tol_eom;       /* EOM: packed residual norm */
  double tol_lin;       /* Lambda and zeta equations: max |residual| */
  double tol_degen;     /* |omega_l - omega_k| below this -> CCSD_ERR_DEGENERATE */
  int max_iter;         /* per solver */
  int diis_dim;         /* DIIS history length */
  int davidson_block;   /* trial vectors transformed per block (<= 16) */
  int davidson_max_sub; /* subspace size before restart */
  int guess;            /* CCSD_GUESS_MP2 */
  void* stream;         /* cudaStream_t, 0 = default */
  double tc_min_flops;  /* contractions below this many flops stay FP64 DFMA (default 1e8) */
  int refine;           /* mixed mode: 1 = refine every solve to the FP64 tolerances above (FP64 residuals
                           with mixed-precision correction solves); 0 = stop at the mixed-precision floor */
  double tol_switch;    /* mixed mode with refine: residual level at which the FP64 refinement starts */
  int autotune;         /* mixed mode: 1 = time the tensor-core tile widths and split counts once per GEMM
                           shape and keep the fastest; 0 = choose them from the output width */
  int fp64_tc;          /* mixed mode: what the handle evaluates at FP64 accuracy (refinement residuals,
                           Hamiltonian-only intermediates, densities) runs its contractions above
                           tc_min_flops as FP64-grade tensor-core products (1, default: 7 fixed-point
                           bf16 slices per operand, exact FP32 sums per K chunk, integer accumulation;
                           error about 2^-46 max|A_m.| max|B_n.| per K term) or as FP64 DFMA (0) */
  /* Device memory: when alloc and free are both set, every device allocation the handle
   * makes (at creation, in its calls and for its caches) goes through them; both NULL (the
   * default): the CUDA runtime (cudaMalloc / cudaMallocAsync); one of them NULL: CCSD_ERR_ARG.
   * alloc(bytes, stream, alloc_ctx) returns memory of the handle's GPU that work queued on
   * `stream` (the handle's stream, as cudaStream_t) after the call may use, or NULL if it
   * cannot, in which case the call that needed it returns CCSD_ERR_OOM and the handle stays
   * usable; free(p, stream, alloc_ctx) releases p once the work already queued on `stream`
   * has finished (the ordering of cudaFreeAsync).  Every block is freed by ccsd_destroy at
   * the latest.  The callbacks are called from the thread making the library call.  Handles
   * with callbacks cannot join a batch (ccsd_batch_create returns CCSD_ERR_ARG). */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_ctx);
  void (*free)(void* p, void* stream, void* alloc_ctx);
  void* alloc_ctx;
} ccsd_options;

/* Fill *opt with defaults (FP64, tol_res 1e-10, tol_eom 1e-7, tol_lin 1e-9, ...). */
void ccsd_default_options(ccsd_options* opt);

/* Create a handle for the Hamiltonian (eps, h, B) with o occupied and v virtual
 * orbitals and naux Cholesky vectors.  Copies the inputs to the device, checks
 * that h and every B^J are symmetric (1e-10, else CCSD_ERR_ARG) and builds the
 * Hamiltonian-only intermediates (the bare vvvv, ovvv and ovov integral blocks).
 * opt may be NULL (defaults).  On failure *out is NULL. */
ccsd_status ccsd_create(const double* eps, const double* h, const double* B, int o, int v, int naux,
                        const ccsd_options* opt, ccsd_handle* out);

/* Solve Omega(t) = 0 (Theory section, amplitude equations) by DIIS-accelerated
 * Jacobi iterations from the MP2-like guess t = -Omega(0)/D.  Also solves the
 * ground-state multipliers lambda^T A = -eta^T.  Returns E_CCSD (total
 * electronic energy <HF|Hbar|HF>) and the iteration count (either may be NULL). */
ccsd_status ccsd_solve_ground(ccsd_handle h, double* e_ccsd, int* iters);

/* Lowest nroots roots (by real part) of A R = omega R (right) with block
 * Davidson; omega[nroots] output (may be NULL).  R_k is normalised to unit
 * packed norm with its largest-magnitude component positive, and
 * R_0^k = eta^T R_k / omega_k. */
ccsd_status eom_solve_right(ccsd_handle h, int nroots, double* omega, int* iters);
/* Left states L_k^T A = omega_k L_k^T for the same nroots; afterwards the left
 * states are biorthonormalised against the right ones, L_k^T R_l = delta_kl
 * (Eq. for the states, L_0^k = 0).  Requires eom_solve_right first. */
ccsd_status eom_solve_left(ccsd_handle h, int nroots, double* omega, int* iters);

/* One block Jacobian transformation at the converged amplitudes:
 * side 0: y_i = A x_i; side 1: y_i = (x_i^T A)^T (Eq. for A), for i < nvec.
 * x, y: [nvec][dim] (host or device).  Host vectors pass through device staging
 * buffers that the handle keeps (grown to the largest block seen) until ccsd_destroy. */
ccsd_status ccsd_jacobian_transform(ccsd_handle h, int side, int nvec, const double* x, double* y);

/* Residual Omega(t) and energy at amplitudes t[dim] (no convergence implied).
 * omega[dim] output; e may be NULL. */
ccsd_status ccsd_residual(ccsd_handle h, const double* t, double* omega, double* e);

/* Restore amplitudes (checkpoint / warm start): t[dim] becomes the ground-state
 * amplitude vector used by the transforms and couplings, as if ccsd_solve_ground
 * had converged to it; lambda[dim] (may be NULL) restores the ground
 * multipliers, otherwise they are solved for.  Returns the energy at t in *e
 * (may be NULL).  Invalidates EOM states.  No convergence check is made on t. */
ccsd_status ccsd_set_amplitudes(ccsd_handle h, const double* t, const double* lambda, double* e);

/* Copy out the converged amplitudes t[dim], the ground multipliers lambda[dim],
 * and EOM states right[k][dim] / left[k][dim] (NULL pointers are skipped). */
ccsd_status ccsd_get_amplitudes(ccsd_handle h, double* t, double* lambda);
ccsd_status ccsd_get_states(ccsd_handle h, int nroots, double* r0, double* right, double* left);

/* Coupling densities for the pair (k, l), k != l: the gradient with respect
 * to (h, B) of the Lagrangian's Hamiltonian-dependent part, so that
 * F_kl^x = sum_pq D_pq dh_pq + sum_Jpq Z_Jpq dB_Jpq (Eq. NAC_NC).  D[n*n],
 * Z[naux*n*n] outputs (Z may be NULL).  Solves the zeta equations of Eq.
 * amplituderelax (or uses the closed form for l = 0).  With relax_orbitals = 1
 * the densities also carry the orbital term kappa-bar_ai F^x_ai: kappa-bar solves
 * kappa-bar^T A^HF = -(k-eta)^T (Eq. orbitalrelax) by conjugate gradients, with
 * k-eta = D_ai - D_ia of the pair's one-electron transition density plus the
 * derivative of the amplitude and excited-state conditions along each
 * occupied-virtual orbital rotation; F^x is the derivative of the Fock matrix
 * along (dh, dB), and dh, dB must be given in the Hartree-Fock orbitals of the
 * handle (ccsd_rotate_integrals). */
ccsd_status ccsd_coupling_densities(ccsd_handle h, int k, int l, double* D, double* Z);

/* F[d] = F_kl^x along ndir directions: dh[d][n*n], dB[d][naux*n*n]. */
ccsd_status ccsd_derivative_coupling(ccsd_handle h, int k, int l, int ndir, const double* dh, const double* dB,
                                     double* F);

/* State-energy gradients (Results section: the crossing-point search needs the gradients
 * of the two states besides their coupling).  The densities of the energy Lagrangian of
 * state k, built like the coupling Lagrangian with the state energy in place of the
 * overlap: for k = 0 (ground state) E + lambda.Omega with lambda^T A = -eta^T; for
 * k >= 1, E_k = E_0 + omega_k and omega_k = L_k.(A R_k) is stationary in the
 * biorthonormal L_k, R_k, so E + lambda.Omega + L_k.(A R_k) + zeta.Omega with
 * zeta^T A = -(F(L_k) R_k)^T (the F-matrix of Eq. for F with gamma = L_k and no reference
 * part).  With relax_orbitals = 1 kappa-bar^T A^HF = -(k-eta)^T adds kappa-bar_ai F^x_ai
 * (no overlap term in k-eta).  D[n*n], Z[naux*n*n] (Z may be NULL), host or device.
 * k = 0 needs ccsd_solve_ground, k >= 1 also both EOM solves (CCSD_ERR_STATE otherwise);
 * k beyond the solved roots: CCSD_ERR_ARG. */
ccsd_status ccsd_gradient_densities(ccsd_handle h, int k, double* D, double* Z);

/* g[d] = dE_k/dx along ndir directions dh[d][n*n], dB[d][naux*n*n] (host or device):
 * sum_pq D_pq dh_pq + sum_Jpq Z_Jpq dB_Jpq with the densities of ccsd_gradient_densities. */
ccsd_status ccsd_energy_gradient(ccsd_handle h, int k, int ndir, const double* dh, const double* dB, double* g);

/* Normalisation factor of a left state (Implementation; Numerical examples, the comparison
 * with full CI): N_k^L = 1/|psi_k^L| with <psi_k^L| = <HF|(l0 + L_k) exp(-T) (k = 0: the
 * ground state's left state, l0 = 1 and L = Lambda).  The left state has no component beyond
 * the doubles, so the norm is exact: a_0^2 plus the metric of the biorthonormal bras applied
 * to a_mu = <psi^L|tau_mu|HF>, a_0 = <psi^L|HF>. */
ccsd_status ccsd_left_norm(ccsd_handle h, int k, double* N);

/* The normalised, antisymmetrised coupling of the paper's comparison with normalised (full
 * CI) states, with N^R approximated by 1/N^L:
 * F[d] = (N_k^L / N_l^L F_kl - N_l^L / N_k^L F_lk) / 2 along ndir directions (as
 * ccsd_derivative_coupling; k != l). */
ccsd_status ccsd_normalized_coupling(ccsd_handle h, int k, int l, int ndir, const double* dh, const double* dB,
                                     double* F);

/* One-electron transition density D[n*n], D_pq = <psi_k^L| E_pq |psi_l^R> at the solved
 * states (k != l; k, l = 0 the ground state), the density the orbital-connection term and
 * the orbital multipliers are built from (section on orbital connections; Implementation,
 * k-eta^1).  Host or device memory. */
ccsd_status ccsd_transition_density(ccsd_handle h, int k, int l, double* D);

/* Orbital-connection term of the coupling (section "Significance of orbital connections"):
 * O[d] = sum_rs (D_rs - D_sr)/2 W[d]_rs with D the (k, l) transition density and W[d][n*n]
 * the ket derivative <phi_r|d phi_s/dx_d> of the unmodified orbitals along each of ndir
 * directions (host or device).  With the symmetric connection T = S^(-1/2) the coupling is
 * ccsd_derivative_coupling along the symmetric-connection Hamiltonian derivative plus O; with
 * the natural connection (the library's default reading) the term is absent. */
ccsd_status ccsd_connection_term(ccsd_handle h, int k, int l, int ndir, const double* W, double* O);

/* Branching plane of the excited states k and l (1 <= k, l, k != l) over ndir coordinate
 * directions taken as orthonormal (Results section, the conical-intersection search):
 *   out[0..ndir)        g = grad (E_l - E_k)
 *   out[ndir..2ndir)    h = (E_l - E_k) F_kl  (F_kl of Eq. NAC_NC along each direction)
 *   out[2ndir..3ndir)   G = P grad E_l + 2 (E_l - E_k) g/|g|, with P the projector onto the
 *                       complement of span{g, h}: the Bearpark-Robb-Schlegel direction whose
 *                       zero is a minimum-energy crossing point.
 * out[3*ndir] host or device memory.  Needs the EOM states (CCSD_ERR_STATE otherwise). */
ccsd_status ccsd_branching_plane(ccsd_handle h, int k, int l, int ndir, const double* dh, const double* dB,
                                 double* out);

/* ---- Hartree-Fock orbitals (relaxed mode) -------------------------------------
 * The nearest Hartree-Fock orbitals to the given orthonormal ones: U = exp(K) with
 * K[a][i] = kappa[i][a] = -K[i][a] (occupied-virtual rotations only), kappa solving
 * F(U^T h U, U^T B U)_ia = 0 (closed-shell Fock matrix, Lagrangian section) by
 * Newton-type steps (J d-kappa = -F' with J = dF'/dkappa at the current orbitals,
 * by GMRES with the preconditioner 1/(eps_a - eps_i); J is not symmetric away from
 * the solution) until max |F'_ia| < tol.  Returns
 * U[n*n] and, when not NULL, the rotated integrals h_out[n*n], B_out[naux*n*n].
 * Arrays may be host or device memory.  CCSD_ERR_NOT_CONVERGED after 100 steps. */
ccsd_status ccsd_scf(const double* eps, const double* h, const double* B, int o, int v, int naux, double tol,
                     double* U_out, double* h_out, double* B_out, int* iters);
/* h_out = U^T h U, B_out^J = U^T B^J U (e.g. a perturbation direction taken to the
 * Hartree-Fock orbitals). */
ccsd_status ccsd_rotate_integrals(const double* U, const double* h, const double* B, int o, int v, int naux,
                                  double* h_out, double* B_out);
/* kappa-bar[o*v] ([i][a]) of the pair (k, l) (relax_orbitals = 1 only; computes the pair's
 * densities if needed). */
ccsd_status ccsd_get_orbital_multipliers(ccsd_handle h, int k, int l, double* kbar);

/* ---- learned initial guess for the doubles amplitudes ---------------------
 * A 3 -> 128 -> 128 -> 1 MLP (tanh hidden layers) maps per-element features
 * x_ijab = (t_MP2, D, |(ia|jb)|), t_MP2 = -(ia|jb)/D, D = e_a + e_b - e_i - e_j, to
 * the correction t_CCSD - t_MP2 (an extension to the paper's method: a starting
 * point for the amplitude equations, which does not change the converged result).
 * A model is CCSD_MLP_PARAMS floats: W1[128][3], b1[128], W2[128][128], b2[128],
 * w3[128], b3, then feature mean[3], feature scale[3], target scale.  Training
 * (Adam, mean squared error) and inference run in the library's kernels; inference
 * uses the weights rounded to bf16 with FP32 accumulation.  Arrays may be host or
 * device memory. */
#define CCSD_MLP_PARAMS 17160
/* Train from scratch on n rows X[n][3], T[n] for `steps` minibatches of `batch`
 * rows (learning rate lr, cosine decay); model_out[CCSD_MLP_PARAMS]; *final_loss =
 * mean squared error over the training rows in units of the target scale. */
ccsd_status ccsd_mlp_train(const float* X, const float* T, long long n, int steps, int batch, float lr,
                           unsigned long long seed, float* model_out, float* final_loss);
/* out[n] = model predictions for X[n][3]. */
ccsd_status ccsd_mlp_predict(const float* model, const float* X, long long n, float* out);
/* grad[CCSD_MLP_PARAMS - 7] = gradient of the mean squared error (normalised target
 * units) over all n rows with respect to the trainable weights; *loss = that error.
 * FP32 weights (no bf16 rounding). */
ccsd_status ccsd_mlp_gradient(const float* model, const float* X, const float* T, long long n, float* grad,
                              float* loss);
/* X[o*o*v*v][3] = the features of the handle's Hamiltonian, doubles in [i][j][a][b] order. */
ccsd_status ccsd_guess_features(ccsd_handle h, float* X);
/* Use `model` for the starting doubles of the next ccsd_solve_ground (NULL: the
 * MP2-type start).  The model is copied. */
ccsd_status ccsd_set_guess_model(ccsd_handle h, const float* model);

/* The same network for the multiplier equations x^T A = -rhs^T (Lambda, lambda^T A = -eta^T,
 * and the zeta equations of Eq. amplituderelax and of the state-energy gradients): their
 * start is the Jacobi step x = -rhs/D, whose doubles take the place of t_MP2 in the
 * features (x_2, D, |(ia|jb)|) and are corrected by the model's prediction.  A model for
 * this is trained on converged ground multipliers (CCSD_GUESS_MULTIPLIERS below).  NULL:
 * the Jacobi start.  The converged multipliers do not depend on the start. */
ccsd_status ccsd_set_multiplier_guess_model(ccsd_handle h, const float* model);

enum { CCSD_GUESS_AMPLITUDES = 0, CCSD_GUESS_MULTIPLIERS = 1 };
/* Training rows from the handle's solved ground state: X[o*o*v*v][3] the features of the
 * start and T[o*o*v*v] = converged doubles - start doubles.  which = CCSD_GUESS_AMPLITUDES:
 * start t_MP2, converged t2; CCSD_GUESS_MULTIPLIERS: start -eta/D, converged lambda.
 * Host or device memory; CCSD_ERR_STATE before ccsd_solve_ground. */
ccsd_status ccsd_guess_targets(ccsd_handle h, int which, float* X, float* T);
/* x2[o*o*v*v] (FP64) = the starting doubles a solve would use with `model` (NULL: the plain
 * start t_MP2, or -eta/D for CCSD_GUESS_MULTIPLIERS, which needs the ground state). */
ccsd_status ccsd_guess_doubles(ccsd_handle h, int which, const float* model, double* x2);
/* Iterations of the handle's last ground-state solve, Lambda solve and zeta solve (any
 * pointer may be NULL); with refinement they count the mixed and FP64 iterations together. */
ccsd_status ccsd_solve_iterations(ccsd_handle h, int* ground, int* lambda, int* zeta);

/* ---- batches of systems -----------------------------------------------------
 * Many small systems underuse the GPU one at a time.  A batch groups handles
 * (systems of any o, v, naux) so that the block Jacobian transforms of all of
 * them run as one CUDA graph launch: the transforms of nvec vectors per system
 * are captured once per side (and per set of active systems) and replayed on
 * every later call; inside the graph each system's kernels run on a stream of
 * its own, so the systems' kernels overlap.  The first call for a side runs the
 * transforms without a graph (this also fixes every lazily built cache and, with
 * opt.autotune, the tile choices) and then captures the graph.
 * While a handle belongs to a batch its calls run on a stream the batch created;
 * ccsd_batch_destroy restores the handle's own stream.  The handles must outlive
 * the batch, and no handle of a batch may be used concurrently with a batch call.
 * (An extension of the method's solvers: the paper treats one system at a time.) */
typedef struct ccsd_batch_ctx* ccsd_batch;
/* nsys >= 1 distinct handles; nvec (1..16) trial vectors per system and launch. */
ccsd_status ccsd_batch_create(int nsys, const ccsd_handle* systems, int nvec, ccsd_batch* out);
/* y[s] = A x[s] (side 0) or (x[s]^T A)^T (side 1) for the nvec vectors of system s;
 * x[s], y[s] are [nvec][dim_s] arrays in host or device memory.  Every system needs
 * amplitudes (ccsd_solve_ground or ccsd_set_amplitudes). */
ccsd_status ccsd_batch_transform(ccsd_batch b, int side, const double* const* x, double* const* y);
/* Lockstep block Davidson over all systems for the nroots (<= nvec) lowest roots:
 * per iteration the new trial vectors of every unconverged system are transformed
 * by one graph launch (each system's block padded with zero vectors to nvec).
 * side 0 leaves every handle as eom_solve_right does, side 1 as eom_solve_left
 * (side 0 first).  Under FP64 refinement (mixed precision with opt.refine) the
 * batched phase stops at 10 tol_switch and each system finishes with its own FP64
 * continuation.  omega[nsys*nroots], iters[nsys] (either may be NULL). */
ccsd_status ccsd_batch_eom_solve(ccsd_batch b, int side, int nroots, double* omega, int* iters);
/* Graph launches, graph captures and kernel nodes of the last captured graph. */
ccsd_status ccsd_batch_stats(ccsd_batch b, long long* launches, long long* captures, long long* nodes);
const char* ccsd_batch_last_error(ccsd_batch b);
void ccsd_batch_destroy(ccsd_batch b);

/* Budget of every pipeline wait (TMA copy, MMA completion, accumulator hand-off) of the
 * handle's tensor-core kernels, in GPU clock cycles; 0 restores the default (4e9 cycles,
 * about 2 s).  A kernel whose wait runs out raises a device flag, waits (with the default
 * bound) for its own copies and MMAs in flight, releases its tensor memory and exits; the
 * call that launched it returns CCSD_ERR_TIMEOUT, and the handle stays usable.  The paper
 * has no counterpart (failure detection of this library).  cycles < 0: CCSD_ERR_ARG. */
ccsd_status ccsd_set_wait_budget(ccsd_handle h, long long cycles);

/* Failure injection for tests of the timeout path (no counterpart in the paper): the next
 * split-bf16 tensor-core GEMM the handle launches issues no operand loads, so the waits of
 * its MMA issuer run out after the wait budget and the call returns CCSD_ERR_TIMEOUT.
 * Nothing is left in flight, no fault is raised, and later calls run normally.  Only for
 * CCSD_PREC_MIXED handles (CCSD_ERR_STATE otherwise). */
ccsd_status ccsd_inject_stall(ccsd_handle h);

/* Allocation-free variant of ccsd_derivative_coupling (the paper has no
 * counterpart; this is a service for callers that cannot allocate device
 * memory at this point, e.g. a dynamics loop running inside a memory pool owned
 * by another framework, or one that must not touch the allocator between time
 * steps because an allocation can synchronise the device).
 * F[d] = sum_pq D_pq dh[d]_pq + sum_Jpq Z_Jpq dB[d]_Jpq with the densities the
 * handle already holds: call ccsd_coupling_densities(h, k, l, ...) first,
 * otherwise CCSD_ERR_STATE.  dh[ndir][n*n] and dB[ndir][naux*n*n] must be device
 * memory of the handle's GPU (the one current at ccsd_create; CCSD_ERR_ARG
 * otherwise); F[ndir] may be host or device memory.
 * 1 <= ndir <= 256 (CCSD_ERR_ARG otherwise).
 * Allocates nothing: the reduction scratch is a fixed 16 KiB array in the
 * library's device image (one per GPU that loads the library, kept until the
 * process exits).  Its device address is looked up on the first call made for
 * each device, with the handle's device made current for the call (the
 * caller's current device is restored on return).  All calls share the array, so calls whose GPU work
 * overlaps (different streams or threads) race and may return wrong values;
 * serialise them.  Launches 4 * ndir + 1 kernels on the handle's stream and
 * synchronises that stream before returning. */
ccsd_status ccsd_derivative_coupling_noalloc(ccsd_handle h, int k, int l, int ndir, const double* dh,
                                             const double* dB, double* F);

/* Counters of the handle's executor since creation: algorithmic flops and calls of the
 * FP64 DFMA GEMMs (flops_fp64, gemms) and of the tensor-core contractions, split-bf16
 * and FP64-grade alike (flops_tc, tc_gemms); any pointer may be NULL. */
ccsd_status ccsd_stats(ccsd_handle h, double* flops_fp64, double* flops_tc, long long* gemms, long long* tc_gemms);

/* One plain contraction C = alpha A B^T + beta C in one of the library's arithmetic forms,
 * for tests and measurements: A (M x K), B (N x K) and C (M x N) are row-major HOST
 * arrays (copied to and from the device; C read only when beta != 0).  form:
 *   CCSD_GEMM_FP64     FP64 DFMA GEMM;
 *   CCSD_GEMM_SPLIT    split-bf16 tensor-core products (splits 2 or 3, FP32 accumulation);
 *   CCSD_GEMM_FP64_TC  FP64-grade tensor-core products (fixed-point slices, see fp64_tc).
 * beta must be 0 or 1 for the tensor-core forms.  reps > 1 repeats the device GEMM reps
 * times (inputs resident) and *ms (may be NULL) receives the mean device time of one, from
 * CUDA events; operand preparation (slicing) is inside the timed region.  Errors:
 * CCSD_ERR_ARG (sizes, form, beta), CCSD_ERR_OOM, CCSD_ERR_CUDA, CCSD_ERR_TIMEOUT. */
enum { CCSD_GEMM_FP64 = 0, CCSD_GEMM_SPLIT = 1, CCSD_GEMM_FP64_TC = 2 };
ccsd_status ccsd_gemm(int form, int splits, int M, int N, int K, double alpha, const double* A, const double* B,
                      double beta, double* C, int reps, double* ms);

/* Kernel-level profile of the calls made between ccsd_profile_start and
 * ccsd_profile_stop: every GEMM launch is bracketed by CUDA events on the
 * handle's stream (small overhead, no extra synchronisation until stop).
 * flops are algorithmic (2 M N K per contraction); tc_issued_flops are the
 * tensor-core MMA flops actually issued (split products and padding).  The
 * "top" fields cover the largest tensor-core contraction (the pp-ladder). */
typedef struct {
  long long launches;         /* kernels launched by the library */
  long long tc_launches;      /* tcgen05 GEMM launches */
  double tc_ms, tc_flops, tc_issued_flops;
  long long fp64_launches;    /* FP64 GEMM launches */
  double fp64_ms, fp64_flops;
  long long top_launches;
  double top_ms, top_flops, top_issued_flops;
  long long ladder_launches;  /* particle-particle ladder GEMMs (two per ladder contraction) */
  double ladder_ms, ladder_flops, ladder_issued_flops;
} ccsd_profile_data;
ccsd_status ccsd_profile_start(ccsd_handle h);
ccsd_status ccsd_profile_stop(ccsd_handle h, ccsd_profile_data* out);

/* One GEMM launch of the last profile (between ccsd_profile_start and ccsd_profile_stop),
 * in launch order: the contraction of the library's tensor program it ran, the arithmetic
 * form, the GEMM shape (batch x M x N x K after the contraction's labels are grouped), the
 * device time from the CUDA events around it (operand slicing included for the tensor-core
 * forms), the algorithmic flops 2 batch M N K and the flops issued (split products and
 * padding included).  The particle-particle ladder runs as two pair-packed GEMMs (+ and -
 * pair combinations, Mp x v(v+1)/2 x v(v+1)/2), each a record with ladder = 1. */
typedef struct {
  char label[160];            /* out[labels] += a[labels] * b[labels], truncated, NUL-terminated */
  int engine;                 /* CCSD_GEMM_FP64, CCSD_GEMM_SPLIT or CCSD_GEMM_FP64_TC */
  int ladder;
  long long batch, m, n, k;
  double ms, flops, issued_flops;
} ccsd_profile_record;

/* Copies min(max, count) records of the last ccsd_profile_stop into out (host memory; out
 * may be NULL when max is 0) and sets *count to the number there are.  Errors: CCSD_ERR_ARG
 * (count NULL, max < 0, out NULL with max > 0). */
ccsd_status ccsd_profile_records(ccsd_handle h, ccsd_profile_record* out, int max, int* count);

const char* ccsd_strerror(ccsd_status s);
const char* ccsd_last_error(ccsd_handle h);
void ccsd_destroy(ccsd_handle h);

/* Host-only: text description of one of the library's tensor programs
 * ("fwd", "jvp", "vjp", "hvp", "dens1", "dens0", and the orbital-relaxation programs
 * "hf_fock", "hf_A", "hf_rotT", "hf_kdens", "hf_rotate").  Writes at most len bytes
 * (NUL-terminated) and returns the full length needed (without the NUL), or
 * -1 for an unknown name.  Touches no GPU. */
long long ccsd_describe_program(const char* which, char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* CCSD_GB300_H */
