"""FP64-grade tensor-core products (fixed-point bf16 slices, exact chunk sums) against FP64.

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
