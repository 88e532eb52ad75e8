"""The FP64 (DFMA) GEMM path's special shapes against numpy FP64, through ccsd_gemm.

C = alpha A B^T + beta C is evaluated by the library in FP64 with a different summation
order than numpy, so each element agrees to a few units of rounding of sum_k |A_mk B_nk|:
the bound tested is 1e-14 K max|A_m.| max|B_n.|.  The shapes cover the skinny kernel (N or M
at most 16 with many rows: one block per row, K split over its threads; the roles of A and B
swapped when M is the small side), the matrix-vector and rank-1 kernels and the tiled kernel
beside them.
"""
import numpy as np
import pytest

from paper_2301_13264_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(3000, 8, 700), (8, 3000, 700), (5000, 16, 33), (600, 1, 900), (700, 9, 1),
                                   (513, 17, 64), (2000, 3, 20000)])
def test_fp64_gemm_shapes(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.normal(size=(M, K))
    Bm = rng.normal(size=(N, K))
    C0 = rng.normal(size=(M, N))
    C, _ = B.ccsd_gemm(B.GEMM_FP64, A, Bm, C=C0.copy(), alpha=0.6, beta=1.0)
    ref = 0.6 * (A @ Bm.T) + C0
    bound = 1e-14 * K * np.abs(A).max(1)[:, None] * np.abs(Bm).max(1)[None, :] + 1e-15 * np.abs(C0)
    assert np.all(np.abs(C - ref) <= bound), (np.abs(C - ref) / bound).max()
    # beta = 0 writes without reading C
    C2, _ = B.ccsd_gemm(B.GEMM_FP64, A, Bm, C=np.full((M, N), np.nan), alpha=1.0, beta=0.0)
    assert np.all(np.abs(C2 - A @ Bm.T) <= bound)
