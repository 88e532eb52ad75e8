"""Pins of the CPU oracle against things other than itself.

* determinant-space evaluation of the paper's definitions (Theory section:
  Hbar, <mu~|, A, eta, F-matrix, Hamiltonian derivatives);
* exact full CI for two electrons, where CCSD is exact (the FCI comparison of
  the numerical examples, with the state normalisation removed exactly);
* finite differences of the definition of the coupling, Eq. (nac);
* the one-body limit (no two-electron integrals), a textbook closed form;
* algebraic invariants: biorthonormality, stationarity of the closed-form
  multipliers (Eq. for gamma), adjointness, orbital-rotation invariance.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle.fockspace import CCBruteForce
from oracle.solvers import State, System, Vec
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes


def T(x):
    return cc.as_t(x)


def maxerr(a, b):
    return max(float(np.abs(np.asarray(x) - np.asarray(y)).max()) for x, y in zip(a, b))


@pytest.mark.parametrize("o,v", [(1, 3), (2, 3), (3, 3)])
def test_residual_and_energy_match_determinant_space(o, v):
    H = make_hamiltonian(o, v, 7, seed=3)
    bf = CCBruteForce(H.h, H.B, o)
    x1, x2 = random_amplitudes(o, v, 5, scale=0.1)
    b1, b2, be = bf.residual(x1[0], x2[0])
    c1, c2, ce = cc.residual(T(x1[0]), T(x2[0]), T(H.h), T(H.B), o)
    assert maxerr((b1, b2), (c1, c2)) < 1e-13
    assert abs(be - float(ce)) < 1e-12
    # t = 0: <HF|H|HF> = sum_i (h_ii + F_ii) fixes the Fock matrix reading
    z1, z2 = np.zeros((o, v)), np.zeros((o, o, v, v))
    b1, b2, be = bf.residual(z1, z2)
    c1, c2, ce = cc.residual(T(z1), T(z2), T(H.h), T(H.B), o)
    assert abs(be - float(ce)) < 1e-12
    assert maxerr((b1, b2), (c1, c2)) < 1e-13


def test_vvvv_batching_is_exact():
    o, v = 2, 7
    H = make_hamiltonian(o, v, 9, seed=4)
    x1, x2 = random_amplitudes(o, v, 1, scale=0.1)
    a = cc.residual(T(x1[0]), T(x2[0]), T(H.h), T(H.B), o)
    b = cc.residual(T(x1[0]), T(x2[0]), T(H.h), T(H.B), o, vvvv_batch=3)
    assert maxerr(a[:2], b[:2]) < 1e-15


@pytest.mark.parametrize("o,v", [(2, 3), (3, 3)])
def test_derivatives_match_determinant_space(o, v):
    H = make_hamiltonian(o, v, 7, seed=3)
    bf = CCBruteForce(H.h, H.B, o)
    X1, X2 = random_amplitudes(o, v, 5, scale=0.1, nvec=4)
    t1, t2, r1, r2, l1, l2, g1, g2 = X1[0], X2[0], X1[1], X2[1], X1[2], X2[2], X1[3], X2[3]
    h, B = T(H.h), T(H.B)
    tt = (T(t1), T(t2))
    assert maxerr(bf.jacobian_right(t1, t2, r1, r2), cc.jacobian_right(*tt, T(r1), T(r2), h, B, o)) < 1e-13
    assert maxerr(bf.jacobian_left(t1, t2, l1, l2), cc.jacobian_left(*tt, T(l1), T(l2), h, B, o)) < 1e-13
    assert maxerr(bf.eta(t1, t2), cc.eta(*tt, h, B, o)) < 1e-13
    for g0 in (0.0, 0.7):
        b = bf.fmatrix(t1, t2, g0, g1, g2, r1, r2)
        c = cc.lagrangian_hessian_right(*tt, g0, T(g1), T(g2), T(r1), T(r2), h, B, o)
        assert maxerr(b, c) < 1e-13
    Hx = bf.hamiltonian_derivative(H.h1, H.B, H.B1)
    b = bf.residual_x(t1, t2, Hx)
    c = cc.hamiltonian_derivative_residual(*tt, h, B, T(H.h1), T(H.B1), o)
    assert maxerr(b[:2], c[:2]) < 1e-14
    assert abs(b[2] - float(c[2])) < 1e-14


def test_tau_expectation_and_overlap_match_determinant_space():
    o, v = 2, 3
    H = make_hamiltonian(o, v, 7, seed=8)
    bf = CCBruteForce(H.h, H.B, o)
    S = System(H.eps, H.h, H.B, o)
    X1, X2 = random_amplitudes(o, v, 11, scale=0.2, nvec=3)
    L = State(0.4, Vec(T(X1[0]), T(X2[0])))
    R = State(-0.3, Vec(T(X1[1]), T(X2[1])))
    D = Vec(T(X1[2]), T(X2[2]))
    b = bf.tau_expectation(0.4, X1[0], X2[0], -0.3, X1[1], X2[1])
    c = S.tau_expectation(L, R)
    assert maxerr(b, (c.x1, c.x2)) < 1e-14
    b = bf.overlap_shifted(0.4, X1[0], X2[0], -0.3, X1[1], X2[1], X1[2], X2[2])
    assert abs(b - float(S.overlap(L, R, D))) < 1e-14


@pytest.fixture(scope="module")
def two_electron():
    o, v = 1, 5
    H = make_hamiltonian(o, v, 6, seed=2)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(3, dense=True, tol=1e-12, tol_lin=1e-12)
    bf = CCBruteForce(H.h, H.B, o)
    return H, S, res, bf


def test_two_electron_energies_equal_fci(two_electron):
    H, S, res, bf = two_electron
    w, U = bf.fci()
    assert abs(res.e_ccsd - w[0]) < 1e-10
    assert np.abs(np.array(res.omega) - (w[1:4] - w[0])).max() < 1e-9


def test_two_electron_couplings_equal_fci(two_electron):
    """c_i F_ij / c_j = <Psi_i|H^x|Psi_j>/(E_j - E_i), c_k = <Psi_k|psi_k^R>.

    For two electrons the CC states are exact, psi_k^R = c_k Psi_k and
    psi_k^L = Psi_k / c_k, so the biorthonormal coupling differs from the FCI
    one only by c_j / c_i (the normalisation factors of the numerical examples).
    """
    H, S, res, bf = two_electron
    o, v = 1, 5
    w, U = bf.fci()
    Hx = bf.hamiltonian_derivative(H.h1, H.B, H.B1)
    t = res.t

    def psi_r(k):
        if k == 0:
            return bf.state_right(t.x1.numpy(), t.x2.numpy(), 1.0, np.zeros((o, v)), np.zeros((o, o, v, v)))
        st = res.right[k - 1]
        return bf.state_right(t.x1.numpy(), t.x2.numpy(), st.c0, st.vec.x1.numpy(), st.vec.x2.numpy())

    c = [U[:, k] @ psi_r(k) for k in range(4)]
    F = {}
    for (i, j) in [(1, 2), (2, 1), (0, 1), (1, 0), (0, 3), (3, 0), (2, 3)]:
        F[(i, j)] = S.coupling(res, i, j, H.h1, H.B1, tol_lin=1e-12)
        ref = U[:, i] @ Hx @ U[:, j] / (w[j] - w[i])
        assert abs(c[i] * F[(i, j)] / c[j] - ref) < 1e-9 * max(abs(ref), 1e-3)
    # normalised couplings are antisymmetric in the exact limit
    for (i, j) in [(1, 2), (0, 1), (0, 3)]:
        a = c[i] * F[(i, j)] / c[j]
        b = c[j] * F[(j, i)] / c[i]
        assert abs(a + b) < 1e-9 * abs(a)


def test_one_body_limit():
    """With B = 0 the exact ground state is a determinant of eigenvectors of h."""
    o, v = 2, 3
    H = make_hamiltonian(o, v, 4, seed=6)
    B0 = np.zeros_like(H.B)
    S = System(H.eps, H.h, B0, o)
    res = S.run(3, dense=True, tol=1e-12)
    lam = np.linalg.eigvalsh(H.h)
    assert abs(res.e_ccsd - 2.0 * lam[:o].sum()) < 1e-10
    # lowest singlet excitation: HOMO -> LUMO of h
    assert abs(res.omega[0] - (lam[o] - lam[o - 1])) < 1e-9
    assert float(res.t.x2.abs().max()) < 1e-10


@pytest.fixture(scope="module")
def small_system():
    o, v = 2, 4
    H = make_hamiltonian(o, v, 8, seed=1)
    S = System(H.eps, H.h, H.B, o)
    res = S.run(3, dense=True, tol=1e-13, tol_lin=1e-13)
    return H, S, res


@pytest.mark.parametrize("i,j", [(1, 2), (2, 1), (0, 1), (1, 0), (0, 2), (2, 0), (3, 1)])
def test_coupling_equals_finite_difference_of_definition(small_system, i, j):
    H, S, res = small_system
    fa = S.coupling(res, i, j, H.h1, H.B1, tol_lin=1e-13)
    fd = S.coupling_fd(res, i, j, H.h1, H.B1, delta=4e-3)
    assert abs(fa - fd) < 1e-6 * abs(fa)


def test_biorthonormality_and_state_invariants(small_system):
    H, S, res = small_system
    t = res.t
    n = len(res.omega)
    for k in range(n):
        for l in range(n):
            assert abs(res.left[k].vec.dot(res.right[l].vec) - (1.0 if k == l else 0.0)) < 1e-10
        # <L_0|R_k> = R0 + lambda^T R_k = 0
        assert abs(res.right[k].c0 + res.lam.dot(res.right[k].vec)) < 1e-10
        # eigen-equations
        r = S.right(t, res.right[k].vec) - res.right[k].vec * res.omega[k]
        l = S.left(t, res.left[k].vec) - res.left[k].vec * res.omega[k]
        assert r.maxabs() < 1e-10 and l.maxabs() < 1e-10
    assert float((t.x2 - t.x2.permute(1, 0, 3, 2)).abs().max()) == 0.0


def test_gamma_multiplier_is_stationary(small_system):
    """L_i + gamma^T (A - omega_j) = 0 with gamma = L_i/(omega_j - omega_i)."""
    H, S, res = small_system
    t = res.t
    i, j = 1, 2
    gam = res.left[i - 1].vec / (res.omega[j - 1] - res.omega[i - 1])
    r = res.left[i - 1].vec + S.left(t, gam) - gam * res.omega[j - 1]
    assert r.maxabs() < 1e-10


def test_adjointness_and_jacobian_is_derivative():
    o, v = 2, 4
    H = make_hamiltonian(o, v, 8, seed=12)
    S = System(H.eps, H.h, H.B, o)
    X1, X2 = random_amplitudes(o, v, 13, scale=0.05, nvec=3)
    t, r, l = (Vec(T(X1[k]), T(X2[k])) for k in range(3))
    ar = S.right(t, r)
    la = S.left(t, l)
    assert abs(l.dot(ar) - la.dot(r)) < 1e-14
    d = 1e-4
    p = S.residual(t + r * d)[0]
    m = S.residual(t - r * d)[0]
    fd = (p - m) / (2 * d)
    assert (fd - ar).maxabs() < 1e-8


def test_fmatrix_is_symmetric_and_the_derivative_of_the_jacobian():
    """F(g) is the second derivative of g0 E + g.Omega: S.(F R) = R.(F S), and S.(F R) equals the
    derivative of g0 eta.R + g.(A(t) R) along S (the F-matrix transformation of Eq. for F)."""
    o, v = 2, 4
    H = make_hamiltonian(o, v, 8, seed=14)
    S = System(H.eps, H.h, H.B, o)
    X1, X2 = random_amplitudes(o, v, 15, scale=0.05, nvec=4)
    t, g, r, s_ = (Vec(T(X1[k]), T(X2[k])) for k in range(4))
    for g0 in (0.0, 0.6):
        fr = S.hess_right(t, g0, g, r)
        fs = S.hess_right(t, g0, g, s_)
        assert abs(s_.dot(fr) - r.dot(fs)) < 1e-14 * max(1.0, abs(s_.dot(fr)))
        d = 1e-4

        def lin(x):
            return g0 * S.eta(x).dot(r) + g.dot(S.right(x, r))

        fd = (lin(t + s_ * d) - lin(t - s_ * d)) / (2 * d)
        assert abs(fd - s_.dot(fr)) < 1e-8 * max(1.0, abs(fd))


def test_davidson_matches_dense(small_system):
    H, S, res = small_system
    omega, R, L = S.eom(res.t, 3, dense=False, tol=1e-10)
    assert np.abs(np.array(omega) - np.array(res.omega)).max() < 1e-10
    for k in range(3):
        assert (R[k].vec - res.right[k].vec).maxabs() < 1e-8
        assert (L[k].vec - res.left[k].vec).maxabs() < 1e-7


def test_orbital_rotation_invariance():
    """E, omega and F_kl F_lk do not change under rotations within the oo and vv blocks.

    F_kl alone scales as s_l/s_k with the state scales, and the packed norm that
    fixes them is not rotation invariant; the product of the two orderings is.
    """
    o, v = 2, 4
    H = make_hamiltonian(o, v, 8, seed=1)
    rng = np.random.default_rng(5)
    Q = np.zeros((o + v, o + v))
    Q[:o, :o] = np.linalg.qr(rng.normal(size=(o, o)))[0]
    Q[o:, o:] = np.linalg.qr(rng.normal(size=(v, v)))[0]
    rot = lambda m: Q.T @ m @ Q
    rotB = lambda b: np.einsum("pq,Ppr,rs->Pqs", Q, b, Q)
    S0 = System(H.eps, H.h, H.B, o)
    S1 = System(H.eps, rot(H.h), rotB(H.B), o)
    r0 = S0.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    r1 = S1.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    assert abs(r0.e_ccsd - r1.e_ccsd) < 1e-10
    assert np.abs(np.array(r0.omega) - np.array(r1.omega)).max() < 1e-9
    for (i, j) in [(1, 2), (0, 1), (0, 2)]:
        p0 = (S0.coupling(r0, i, j, H.h1, H.B1, tol_lin=1e-12)
              * S0.coupling(r0, j, i, H.h1, H.B1, tol_lin=1e-12))
        p1 = (S1.coupling(r1, i, j, rot(H.h1), rotB(H.B1), tol_lin=1e-12)
              * S1.coupling(r1, j, i, rot(H.h1), rotB(H.B1), tol_lin=1e-12))
        assert abs(p0 - p1) < 1e-8 * abs(p0)


def test_davidson_survives_transient_complex_pair():
    """A small Davidson subspace of the non-symmetric left Jacobian gives a complex Ritz pair
    among the wanted roots of this system (o=3, v=6, naux=9, seed 5), although the two lowest
    roots are real.  With no complex expansion allowed the solve fails, which shows the pair
    occurs; with the default rule it converges to the dense diagonalisation's roots and vectors."""
    H = make_hamiltonian(3, 6, 9, seed=5)
    S = System(H.eps, H.h, H.B, 3)
    t, _, _ = S.solve_ground(tol=1e-12)
    with pytest.raises(RuntimeError, match="complex root"):
        S.davidson(lambda x: S.left(t, x), 2, tol=1e-10, max_complex=0)
    omega_d, R_d, L_d = S.eom(t, 2, dense=True)
    omega, R, L = S.eom(t, 2, dense=False, tol=1e-10)
    assert np.abs(np.array(omega) - np.array(omega_d)).max() < 1e-10
    for k in range(2):
        assert (R[k].vec - R_d[k].vec).maxabs() < 1e-8
        assert (L[k].vec - L_d[k].vec).maxabs() < 1e-8
