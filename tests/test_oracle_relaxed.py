"""Pins of the oracle's orbital relaxation (CPU only).

Hartree-Fock orbitals: the rotated Fock matrix has no occupied-virtual block,
the Hartree-Fock energy is stationary under further rotations, and Brillouin's
theorem holds in determinant space.  The transition density equals
<psi^L|E_pq|psi^R> evaluated literally in determinant space.  The relaxed coupling
equals finite differences of the definition with the orbitals re-optimised at every
displacement and the ket mapped back by the many-body rotation operator, and for
two electrons (CCSD = full CI, which does not depend on the orbitals) it equals the
unrelaxed coupling.  The same holds for the state-energy gradients with the orbital
term: finite differences of E_k(x) with re-optimised orbitals, and relaxed = unrelaxed
for two electrons.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle import relaxed as rx
from oracle.fockspace import CCBruteForce
from oracle.solvers import System
from paper_2301_13264_gb300.synth import make_hamiltonian


def _hf_system(o, v, naux, seed, bscale=0.1):
    """A synthetic Hamiltonian rotated to its nearest Hartree-Fock orbitals, with the
    perturbation direction expressed in those orbitals."""
    H = make_hamiltonian(o, v, naux, seed=seed, bscale=bscale)
    _, U, h0, B0 = rx.scf(H.h, H.B, o)
    h1, B1 = rx.rotate(H.h1, H.B1, U)
    return h0.numpy(), B0.numpy(), h1.numpy(), B1.numpy()


def _hf_energy(h, B, o):
    F = rx.fock(h, B, o)
    return float(torch.diagonal(cc.as_t(h)[:o, :o]).sum() + torch.diagonal(F[:o, :o]).sum())


def test_scf_conditions():
    o, v, naux = 2, 4, 9
    H = make_hamiltonian(o, v, naux, seed=3)
    kappa, U, h0, B0 = rx.scf(H.h, H.B, o)
    assert float(kappa.abs().max()) > 1e-3  # the synthetic reference is not Hartree-Fock
    assert torch.allclose(U.T @ U, torch.eye(o + v, dtype=torch.float64), atol=1e-14)
    assert float(rx.fock(h0, B0, o)[:o, o:].abs().max()) < 1e-12
    # stationarity of E_HF = sum_i (h_ii + F_ii) under further occupied-virtual rotations
    rng = np.random.default_rng(1)
    d = torch.as_tensor(rng.normal(size=(o, v)))
    e = lambda s: _hf_energy(*rx.rotate(h0, B0, torch.linalg.matrix_exp(rx.kappa_matrix(s * d, o, o + v))), o)
    s = 1e-3  # central differences with one Richardson step: error O(s^4)
    slope = (8 * (e(s) - e(-s)) - (e(2 * s) - e(-2 * s))) / (12 * s)
    curv = (e(s) - 2 * e(0.0) + e(-s)) / s ** 2
    assert abs(slope) < 1e-10 and curv > 1e-2
    # Brillouin: <Phi_i^a|H|HF> = 0 in determinant space
    bf = CCBruteForce(h0.numpy(), B0.numpy(), o)
    hf = bf.fs.hf_vector()
    Hhf = bf.H @ hf
    for i in range(o):
        for a in range(v):
            assert abs((bf.fs.E(o + a, i) @ hf) @ Hhf) < 1e-11


def test_hf_hessian_symmetric_positive():
    h0, B0, _, _ = _hf_system(2, 5, 11, seed=4)
    A = rx.hf_hessian(h0, B0, 2).numpy()
    assert np.abs(A - A.T).max() < 1e-12
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


@pytest.mark.parametrize("pair", [(0, 0), (1, 2), (2, 1), (0, 1), (1, 0)])
def test_transition_density_against_determinant_space(pair):
    o, v = 2, 3
    h0, B0, _, _ = _hf_system(o, v, 8, seed=5)
    S = System(np.diag(rx.fock(h0, B0, o).numpy()), h0, B0, o)
    res = S.run(2, dense=True, tol=1e-13, tol_lin=1e-13)
    i, j = pair
    L, R = S.left_state(res, i), S.right_state(res, j)
    D = rx.transition_density(S, res, L, R).numpy()
    bf = CCBruteForce(h0, B0, o)
    t = res.t
    bra = bf.state_left(t.x1.numpy(), t.x2.numpy(), L.c0, L.vec.x1.numpy(), L.vec.x2.numpy())
    ket = bf.state_right(t.x1.numpy(), t.x2.numpy(), R.c0, R.vec.x1.numpy(), R.vec.x2.numpy())
    for p in range(o + v):
        for q in range(o + v):
            assert abs(D[p, q] - bra @ (bf.fs.E(p, q) @ ket)) < 1e-11


@pytest.mark.parametrize("pair", [(1, 2), (2, 1), (0, 1), (1, 0), (2, 0)])
def test_relaxed_coupling_equals_finite_differences(pair):
    # strong two-electron integrals, so that CCSD is far enough from full CI for the
    # orbital term to matter (for weak ones CCSD is nearly orbital-invariant here)
    o, v, naux = 2, 3, 8
    h0, B0, h1, B1 = _hf_system(o, v, naux, seed=6, bscale=0.4)
    i, j = pair
    fd, S, res = rx.relaxed_overlap_fd(h0, B0, h1, B1, o, i, j, nroots=2)
    f, kbar = rx.relaxed_coupling(S, res, i, j, h1, B1, tol_lin=1e-13)
    f_unrelaxed = S.coupling(res, i, j, h1, B1, tol_lin=1e-13)
    assert abs(f - fd) < 1e-9
    # the orbital term is resolved: relaxed and unrelaxed couplings differ by far more
    assert abs(f - f_unrelaxed) > 1e-6


def test_two_electrons_relaxed_equals_unrelaxed():
    o, v, naux = 1, 4, 7
    h0, B0, h1, B1 = _hf_system(o, v, naux, seed=7)
    S = System(np.diag(rx.fock(h0, B0, o).numpy()), h0, B0, o)
    res = S.run(3, dense=True, tol=1e-13, tol_lin=1e-13)
    for (i, j) in [(1, 2), (2, 3), (0, 1), (1, 0)]:
        f, _ = rx.relaxed_coupling(S, res, i, j, h1, B1, tol_lin=1e-13)
        f0 = S.coupling(res, i, j, h1, B1, tol_lin=1e-13)
        assert abs(f - f0) < 1e-9 * max(1.0, abs(f0))


@pytest.mark.parametrize("k", [0, 1, 2])
def test_relaxed_energy_gradient_equals_finite_differences(k):
    """dE_k/dx with the orbitals re-optimised at every displacement (energies only, no states
    mapped between orbital sets) against the Lagrangian with the kappa-bar term."""
    o, v, naux = 2, 3, 8
    h0, B0, h1, B1 = _hf_system(o, v, naux, seed=6, bscale=0.4)
    fd, S, res = rx.relaxed_energy_fd(h0, B0, h1, B1, o, k, nroots=2)
    g = rx.relaxed_energy_gradient(S, res, k, h1, B1, tol_lin=1e-13)
    assert abs(g - fd) < 1e-9
    assert abs(g - S.energy_gradient(res, k, h1, B1, tol_lin=1e-13)) > 1e-7


def test_two_electrons_relaxed_energy_gradient_equals_unrelaxed():
    o, v, naux = 1, 4, 7
    h0, B0, h1, B1 = _hf_system(o, v, naux, seed=7)
    S = System(np.diag(rx.fock(h0, B0, o).numpy()), h0, B0, o)
    res = S.run(3, dense=True, tol=1e-13, tol_lin=1e-13)
    for k in range(4):
        g = rx.relaxed_energy_gradient(S, res, k, h1, B1, tol_lin=1e-13)
        assert abs(g - S.energy_gradient(res, k, h1, B1, tol_lin=1e-13)) < 1e-9 * max(1.0, abs(g))
