"""Pins of the oracle's left-state normalisation N^L and the normalised, antisymmetrised
coupling of the paper's comparison with full CI.

* N^L = 1/|<HF|(l0 + L) exp(-T)| against the determinant-space norm of the same bra, for
  converged ground and excited left states and for random amplitudes and left vectors
  (o = 1, 2, 3): the closed form of the biorthonormal-bra metric and the components must both
  be right;
* two electrons, where CC is exact: psi_k^L = Psi_k / c_k with c_k = <Psi_k|psi_k^R>, so
  N_k^L = |c_k| and the normalised coupling equals the full-CI coupling
  <Psi_i|H^x|Psi_j>/(E_j - E_i) up to the sign of c_i c_j.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import normalization as nm
from oracle.fockspace import CCBruteForce
from oracle.solvers import Result, State, System, Vec
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes


@pytest.mark.parametrize("o,v,seed", [(1, 4, 1), (2, 3, 2), (3, 2, 3), (2, 4, 4)])
def test_left_norm_equals_determinant_space(o, v, seed):
    H = make_hamiltonian(o, v, 2 * (o + v), seed=seed)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    bf = CCBruteForce(H.h, H.B, o)
    t = res.t
    for k in range(3):
        L = S.left_state(res, k)
        bra = bf.state_left(t.x1.numpy(), t.x2.numpy(), L.c0, L.vec.x1.numpy(), L.vec.x2.numpy())
        assert abs(nm.left_norm(S, res, k) - 1.0 / np.linalg.norm(bra)) < 1e-13
    # generic amplitudes and left vectors (not solutions): every component of the formula
    X1, X2 = random_amplitudes(o, v, seed + 40, scale=0.3, nvec=2)
    tr = Vec(cc.as_t(X1[0]), cc.as_t(X2[0]))
    for l0 in (0.0, 0.7):
        r = Result(t=tr, lam=Vec(cc.as_t(X1[1]), cc.as_t(X2[1])))
        Lst = State(l0, r.lam)
        r.left = [Lst]
        a0, a = nm.left_components(S, r, 1)
        bra = bf.state_left(X1[0], X2[0], l0, X1[1], X2[1])
        assert abs(nm.bra_metric_norm2(a0, a) - float(bra @ bra)) < 1e-12 * float(bra @ bra)


def test_two_electron_normalized_coupling_equals_fci():
    o, v = 1, 5
    H = make_hamiltonian(o, v, 6, seed=2)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(3, dense=True, tol=1e-12, tol_lin=1e-12)
    bf = CCBruteForce(H.h, H.B, o)
    w, U = bf.fci()
    Hx = bf.hamiltonian_derivative(H.h1, H.B, H.B1)
    t = res.t

    def psi_r(k):
        st = State(1.0, Vec.zeros(o, v)) if k == 0 else res.right[k - 1]
        return bf.state_right(t.x1.numpy(), t.x2.numpy(), st.c0, st.vec.x1.numpy(), st.vec.x2.numpy())

    c = [U[:, k] @ psi_r(k) for k in range(4)]
    for k in range(4):
        assert abs(nm.left_norm(S, res, k) - abs(c[k])) < 1e-10
    for (i, j) in [(1, 2), (0, 1), (0, 3), (2, 3)]:
        ref = U[:, i] @ Hx @ U[:, j] / (w[j] - w[i])
        f = nm.normalized_coupling(S, res, i, j, H.h1, H.B1, tol_lin=1e-12)
        assert abs(f - np.sign(c[i] * c[j]) * ref) < 1e-9 * max(abs(ref), 1e-3), (i, j, f, ref)
