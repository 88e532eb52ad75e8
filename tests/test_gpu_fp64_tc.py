"""FP64-grade tensor-core products (fixed-point bf16 slices, exact chunk sums) against FP64,
as plain GEMMs and as the handle form CCSD_PREC_FP64_TC against the oracle.

The reference is the plain definition C = alpha A B^T + beta C evaluated by numpy in
FP64.  The scheme keeps 49 bits of every operand below its row's leading bit and drops
the slice products of level >= 7, so each K term carries an error of about
2^-46 max_k |A_mk| max_k |B_nk|; the bound tested is 2^-43 K max|A_m.| max|B_n.| per
element.  Integer operands whose products and sums are exact in FP64 give bit-exact
results, and a non-finite operand row gives non-finite outputs in its row or column.
"""
import numpy as np
import pytest

from paper_2301_13264_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-4, 4, (M, 1)))
    Bm = rng.normal(size=(N, K)) * np.exp(rng.uniform(-4, 4, (N, 1)))
    return A, Bm


def _bound(A, Bm):
    K = A.shape[1]
    return 2.0 ** -43 * K * np.abs(A).max(1)[:, None] * np.abs(Bm).max(1)[None, :]


# (M, N, K): one element; ragged tiles; several K chunks; M < 128 (operands swapped);
# few output tiles (split-K); K beyond one split's 28672; many tiles
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (130, 70, 100), (257, 129, 1500), (64, 1000, 3000),
                                   (200, 300, 30000), (1000, 1000, 64)])
def test_matches_fp64(M, N, K):
    A, Bm = _operands(M, N, K, seed=M + N + K)
    C0 = np.random.default_rng(1).normal(size=(M, N))
    ref = -0.7 * (A @ Bm.T) + C0
    C, _ = B.ccsd_gemm(B.GEMM_FP64_TC, A, Bm, C=C0.copy(), alpha=-0.7, beta=1.0)
    err = np.abs(C - ref)
    assert np.all(err <= 0.7 * _bound(A, Bm) + 4e-16 * np.abs(ref)), (err / _bound(A, Bm)).max()
    # far below the split-bf16 products (FP32 accumulation)
    Cs, _ = B.ccsd_gemm(B.GEMM_SPLIT, A, Bm, C=C0.copy(), alpha=-0.7, beta=1.0)
    if K >= 64:
        assert np.linalg.norm(C - ref) < 1e-4 * np.linalg.norm(Cs - ref)


def test_integer_operands_exact():
    rng = np.random.default_rng(7)
    A = rng.integers(-50, 51, (300, 1000)).astype(np.float64)
    Bm = rng.integers(-50, 51, (200, 1000)).astype(np.float64)
    C, _ = B.ccsd_gemm(B.GEMM_FP64_TC, A, Bm)
    assert np.array_equal(C, A @ Bm.T)


def test_zero_and_nonfinite_rows():
    A, Bm = _operands(140, 90, 700, seed=3)
    A[5] = 0.0
    A[17, 33] = np.nan
    Bm[40, 2] = np.inf
    C, _ = B.ccsd_gemm(B.GEMM_FP64_TC, A, Bm)
    assert np.all(C[5][np.arange(90) != 40] == 0.0)
    assert not np.any(np.isfinite(C[17]))
    assert not np.any(np.isfinite(C[:, 40]))
    keep = np.ones(140, bool)
    keep[17] = False
    cols = np.arange(90) != 40
    ref = A[keep] @ Bm[cols].T
    assert np.all(np.abs(C[keep][:, cols] - ref) <= _bound(A[keep], Bm[cols]))


def test_throughput_against_dfma():
    # a particle-particle ladder GEMM at the thymine-dz size, 8 vectors (M = 8 o(o+1)/2, N = K = v(v+1)/2)
    M, N, K = 4488, 7626, 7626
    A, Bm = _operands(M, N, K, seed=5)
    _, ms_tc = B.ccsd_gemm(B.GEMM_FP64_TC, A, Bm, reps=3)
    _, ms_64 = B.ccsd_gemm(B.GEMM_FP64, A, Bm, reps=1)
    tf_tc = 2.0 * M * N * K / ms_tc / 1e9
    tf_64 = 2.0 * M * N * K / ms_64 / 1e9
    print(f"ladder-shaped GEMM {M}x{N}x{K}: FP64-grade tensor cores {ms_tc:.2f} ms ({tf_tc:.1f} TFLOP/s incl. "
          f"slicing), FP64 DFMA {ms_64:.2f} ms ({tf_64:.2f} TFLOP/s)")
    assert ms_tc < ms_64


def _fp64tc_handle(H, **kw):
    o = dict(precision=B.PREC_FP64_TC, tc_min_flops=0.0)
    o.update(kw)
    return B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**o))


@pytest.mark.parametrize("o,v,naux", [(6, 48, 60), (9, 37, 41)])
def test_fp64tc_residual_and_transforms_match_oracle(o, v, naux):
    """Handle form CCSD_PREC_FP64_TC with every contraction on the tensor cores: residual,
    energy and right/left transforms within 1e-11 of the oracle relative to the largest
    element, the bound of the FP64 form (the split-bf16 form is at 2e-5 here)."""
    from oracle import ccsd as cc
    from oracle.solvers import System, Vec
    from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes

    H = make_hamiltonian(o, v, naux, seed=4)
    X1, X2 = random_amplitudes(o, v, 8, scale=0.03, nvec=4)
    flat = lambda a, b: np.concatenate([np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)])  # noqa: E731
    relerr = lambda a, b: np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()  # noqa: E731
    t = flat(X1[0], X2[0])
    h = _fp64tc_handle(H)
    try:
        om = np.zeros_like(t)
        e = B.ccsd_residual(h, t, om)
        assert B.ccsd_stats(h)["tc_gemms"] > 0, "tensor-core path not taken"
        B.ccsd_set_amplitudes(h, t, np.zeros_like(t))
        X = np.stack([flat(X1[k], X2[k]) for k in (1, 2, 3)])
        YR, YL = np.zeros_like(X), np.zeros_like(X)
        B.ccsd_jacobian_transform(h, 0, 3, X, YR)
        B.ccsd_jacobian_transform(h, 1, 3, X, YL)
    finally:
        B.ccsd_destroy(h)
    c1, c2, ce = cc.residual(cc.as_t(X1[0]), cc.as_t(X2[0]), cc.as_t(H.h), cc.as_t(H.B), o)
    assert relerr(om, flat(c1, c2)) < 1e-11
    assert abs(e - float(ce)) < 1e-11 * abs(float(ce))
    S_ = System(H.eps, H.h, H.B, o)
    tv = Vec(cc.as_t(X1[0]), cc.as_t(X2[0]))
    for k in range(3):
        r = Vec(cc.as_t(X1[k + 1]), cc.as_t(X2[k + 1]))
        ar, la = S_.right(tv, r), S_.left(tv, r)
        assert relerr(YR[k], flat(ar.x1, ar.x2)) < 1e-11
        assert relerr(YL[k], flat(la.x1, la.x2)) < 1e-11


def test_fp64tc_pipeline_meets_fp64_tolerances():
    """The whole pipeline in the FP64-grade tensor-core form, solved directly to the FP64
    tolerances: energy within 1e-9 Eh of the oracle, excitation energies within 1e-8,
    couplings within 1e-7 relative."""
    from oracle.solvers import System
    from paper_2301_13264_gb300.synth import workload

    H = workload("small")
    S_ = System(H.eps, H.h, H.B, H.o)
    res = S_.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    h = _fp64tc_handle(H, tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)
    try:
        e, _ = B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        F = {kl: B.ccsd_derivative_coupling(h, kl[0], kl[1], 1, H.h1, H.B1)[0] for kl in [(1, 2), (0, 1), (2, 0)]}
        assert B.ccsd_stats(h)["tc_gemms"] > 0
    finally:
        B.ccsd_destroy(h)
    assert abs(e - res.e_ccsd) < 1e-9
    assert np.abs(np.array(w) - np.array(res.omega)).max() < 1e-8
    for (k, l), f in F.items():
        ref = S_.coupling(res, k, l, H.h1, H.B1, tol_lin=1e-12)
        assert abs(f - ref) < 1e-7 * abs(ref)

