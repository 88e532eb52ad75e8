"""Pins of the oracle's state-energy gradients dE_k/dx (ground and EOM states).

* two electrons, where CCSD and EOM-CCSD are exact: dE_k/dx equals the Hellmann-Feynman
  value <Psi_k|H^x|Psi_k> of the full-CI eigenvector;
* more electrons: central finite differences (one Richardson step) of E_k(x) solved at
  displaced Hamiltonians, the root followed by its overlap with L_k(x0).
"""
import numpy as np
import pytest

from oracle.fockspace import CCBruteForce
from oracle.solvers import System
from paper_2301_13264_gb300.synth import make_hamiltonian


def test_two_electron_gradients_equal_hellmann_feynman():
    o, v = 1, 5
    H = make_hamiltonian(o, v, 6, seed=2)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(3, dense=True, tol=1e-12, tol_lin=1e-12)
    bf = CCBruteForce(H.h, H.B, o)
    w, U = bf.fci()
    Hx = bf.hamiltonian_derivative(H.h1, H.B, H.B1)
    for k in range(4):
        ref = U[:, k] @ Hx @ U[:, k]
        g = S.energy_gradient(res, k, H.h1, H.B1, tol_lin=1e-12)
        assert abs(g - ref) < 1e-9 * max(1.0, abs(ref)), (k, g, ref)


@pytest.mark.parametrize("o,v,naux,seed", [(2, 4, 8, 5), (3, 3, 7, 6)])
def test_gradients_match_finite_differences(o, v, naux, seed):
    H = make_hamiltonian(o, v, naux, seed=seed)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    for k in range(3):
        g = S.energy_gradient(res, k, H.h1, H.B1, tol_lin=1e-12)
        fd = S.energy_gradient_fd(res, k, H.h1, H.B1)
        assert abs(g - fd) < 1e-7 * max(1.0, abs(fd)), (k, g, fd)
    # the excited-state part is not trivially the ground-state one
    assert abs(S.energy_gradient(res, 1, H.h1, H.B1) - S.energy_gradient(res, 0, H.h1, H.B1)) > 1e-4
