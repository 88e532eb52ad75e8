"""Left-state normalisation and the normalised, antisymmetrised coupling on the GPU against
the oracle, whose N^L is pinned to the determinant-space norm and, for two electrons, its
normalised coupling to full CI (tests/test_oracle_normalization.py)."""
import numpy as np
import pytest
import torch

from oracle import normalization as nm
from oracle.solvers import System
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, workload

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available()
    B.lib()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_left_norms_and_normalized_couplings_match_oracle(form):
    H = workload("small")
    S = System(H.eps, H.h, H.B, H.o)
    res = S.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    kw = dict(TIGHT)
    if form == "mixed":
        kw.update(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0, refine=1)
    h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**kw))
    try:
        B.ccsd_solve_ground(h)
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        N = [B.ccsd_left_norm(h, k) for k in range(3)]
        F = {kl: B.ccsd_normalized_coupling(h, kl[0], kl[1], 1, H.h1, H.B1)[0] for kl in [(1, 2), (0, 1), (0, 2)]}
        F21 = B.ccsd_normalized_coupling(h, 2, 1, 1, H.h1, H.B1)[0]
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_left_norm(h, 3)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    for k in range(3):
        ref = nm.left_norm(S, res, k)
        # N^L depends on the eigenvectors to first order: within the EOM residual threshold
        assert abs(N[k] - ref) < 1e-8 * ref, (k, N[k], ref)
    for (i, j), f in F.items():
        ref = nm.normalized_coupling(S, res, i, j, H.h1, H.B1, tol_lin=1e-12)
        assert abs(f - ref) < 1e-7 * abs(ref), (i, j, f, ref)
    # antisymmetric by construction
    assert abs(F21 + F[(1, 2)]) < 1e-12 * abs(F[(1, 2)])
    # the normalisation is not trivial here: the factors differ from 1 by more than the tolerance
    assert max(abs(n - 1.0) for n in N) > 1e-3
