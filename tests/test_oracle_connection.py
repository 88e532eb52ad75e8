"""Pins of the oracle's orbital-connection term (symmetric connection) against finite
differences of the definition.

The coupling is d/dx <psi_i^L(x0)|psi_j^R(x)>; with the symmetric connection the states at x
live in the orbitals psi(x) = S(x)^(-1/2) phi(x), which differ from the x0 orbitals to first
order by Y = (W - W^T)/2.  The oracle's analytic value (Eq. NAC_NC with the symmetric-connection
Hamiltonian derivative, plus sum_rs (D_rs - D_sr)/2 W_rs) must equal central differences of
the definition evaluated in determinant space, where the ket at x is carried into the x0
orbitals by the many-body operator of the orbital overlap.  Dropping the overlap term, or
antisymmetrising the density with the wrong sign, misses by far more than the tolerance.
"""
import numpy as np
import pytest

from oracle import connection as cn
from oracle.solvers import System
from paper_2301_13264_gb300.synth import make_hamiltonian


def ket_derivative(n, seed, scale=0.05):
    """A ket-derivative matrix W with symmetric and antisymmetric parts."""
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(n, n))


@pytest.mark.parametrize("o,v,naux,seed", [(1, 3, 5, 21), (2, 3, 6, 22)])
def test_symmetric_connection_coupling_equals_finite_differences(o, v, naux, seed):
    H = make_hamiltonian(o, v, naux, seed=seed)
    W = ket_derivative(o + v, seed)
    for (i, j) in [(1, 2), (2, 1), (0, 1), (2, 0)]:
        fd, S, res = cn.symmetric_connection_fd(H.eps, H.h, H.B, H.h1, H.B1, W, o, i, j, nroots=2)
        f = cn.symmetric_connection_coupling(S, res, i, j, H.h1, H.B1, W, tol_lin=1e-13)
        term = cn.connection_term(S, res, i, j, W)
        assert abs(f - fd) < 1e-7 * max(1.0, abs(fd)), (i, j, f, fd)
        # the overlap term is resolved: without it, or with the density symmetrised, the value misses
        assert abs(term) > 1e3 * abs(f - fd)


def test_connection_term_vanishes_for_a_symmetric_ket_derivative():
    """W = W^T (an overlap that only scales the orbitals symmetrically): Y = 0, no term."""
    o, v = 2, 3
    H = make_hamiltonian(o, v, 6, seed=23)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(2, dense=True, tol=1e-13, tol_lin=1e-13)
    W = ket_derivative(o + v, 5)
    assert abs(cn.connection_term(S, res, 1, 2, W + W.T)) < 1e-14
    assert abs(cn.connection_term(S, res, 1, 2, W - W.T)) > 1e-4
