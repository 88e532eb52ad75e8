"""Orbital-connection term and transition density on the GPU against the oracle.

The oracle's symmetric-connection coupling (Eq. NAC_NC along the symmetric-connection
Hamiltonian derivative plus sum_rs (D_rs - D_sr)/2 W_rs) is pinned to finite differences of
the definition in determinant space (tests/test_oracle_connection.py), its transition density
to <psi^L|E_pq|psi^R> in determinant space (tests/test_oracle_relaxed.py).  The directions
(dh^sym, dB^sym) are Hamiltonian derivatives, inputs of the method; the test prepares them with
the oracle's helper and gives them to the library like any other direction.
"""
import numpy as np
import pytest
import torch

from oracle import connection as cn
from oracle import relaxed as rx
from oracle.solvers import System
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)
PAIRS = [(1, 2), (2, 1), (0, 1), (2, 0)]


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available()
    B.lib()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_connection_term_and_symmetric_coupling_match_oracle(form):
    o, v, naux = 3, 8, 14
    H = make_hamiltonian(o, v, naux, seed=31)
    n = o + v
    rng = np.random.default_rng(32)
    W = np.ascontiguousarray(np.stack([0.05 * rng.normal(size=(n, n)), 0.05 * rng.normal(size=(n, n))]))
    S = System(H.eps, H.h, H.B, o)
    res = S.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    dsym = [cn.symmetric_connection_derivatives(S.h, S.B, H.h1, H.B1, W[d]) for d in range(2)]
    dh = np.ascontiguousarray(np.stack([x[0].numpy() for x in dsym]))
    dB = np.ascontiguousarray(np.stack([x[1].numpy() for x in dsym]))
    kw = dict(TIGHT)
    if form == "mixed":
        kw.update(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0, refine=1)
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, B.ccsd_default_options(**kw))
    got = {}
    try:
        B.ccsd_solve_ground(h)
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        for kl in PAIRS:
            D = np.zeros((n, n))
            B.ccsd_transition_density(h, kl[0], kl[1], D)
            term = B.ccsd_connection_term(h, kl[0], kl[1], 2, torch.as_tensor(W, device="cuda"))
            F = B.ccsd_derivative_coupling(h, kl[0], kl[1], 2, dh, dB)
            got[kl] = (D, term, [F[d] + term[d] for d in range(2)])
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_connection_term(h, 1, 1, 2, W)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    for kl in PAIRS:
        D, term, Fsym = got[kl]
        Dref = rx.transition_density(S, res, S.left_state(res, kl[0]), S.right_state(res, kl[1])).numpy()
        assert np.abs(D - Dref).max() < 1e-8 * np.abs(Dref).max(), kl
        for d in range(2):
            tref = cn.connection_term(S, res, kl[0], kl[1], W[d])
            fref = cn.symmetric_connection_coupling(S, res, kl[0], kl[1], H.h1, H.B1, W[d], tol_lin=1e-12)
            assert abs(term[d] - tref) < 1e-7 * abs(tref) + 1e-10, (kl, d, term[d], tref)
            assert abs(Fsym[d] - fref) < 1e-7 * abs(fref) + 1e-10, (kl, d, Fsym[d], fref)
            # the term is a sizeable part of the symmetric-connection coupling
            assert abs(tref) > 1e-3 * abs(fref)
