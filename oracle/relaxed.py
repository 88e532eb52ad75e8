"""Orbital relaxation: Hartree-Fock orbitals that follow x, and the relaxed coupling (oracle).

Test infrastructure of the oracle; see the package docstring.

The Lagrangian of the Theory section carries the Hartree-Fock conditions F_ai = 0
with multipliers kappa-bar.  Stationarity in the orbital rotation parameters
kappa gives kappa-bar^T A^HF = -(k-eta)^T (Eq. orbitalrelax), with k-eta the
kappa-derivative of the overlap term plus that of the amplitude and
excited-state conditions, and the coupling gains kappa-bar_ai F^q_ai
(Eq. NAC_NC); the first term of k-eta is D_ai - D_ia of the one-electron
transition density (Implementation section).

Conventions (written out here because the paper leaves them to its program):
* orbitals rotate by U(kappa) = exp(K) with occupied-virtual generators only,
  K[a, i] = kappa[i, a], K[i, a] = -kappa[i, a] (kappa stored [i][a] like t1);
* rotated integrals h' = U^T h U and B'^J = U^T B^J U; a state built from them is,
  in the original orbitals, exp(sum_rs K_rs E_rs) applied to it;
* the Hartree-Fock orbitals at x are the ones reached from the x0 orbitals by
  such a rotation (the nearest Hartree-Fock solution, no occupied-occupied or
  virtual-virtual mixing); at x0 the orbitals are Hartree-Fock, kappa(x0) = 0;
* A^HF[ai, bj] = dF'_ai / dkappa_bj at kappa = 0 (F' the Fock matrix of the
  rotated integrals), so that kappa-bar^T A^HF = -(k-eta)^T with k-eta_ai the
  derivative of the rest of the Lagrangian with respect to kappa_ai.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import torch

from . import ccsd as cc
from .solvers import State, System, Vec

F64 = torch.float64


def kappa_matrix(kappa, o: int, n: int):
    """Antisymmetric generator K for kappa[o][v]."""
    kappa = cc.as_t(kappa)
    K = torch.zeros((n, n), dtype=F64)
    K[o:, :o] = kappa.T
    K[:o, o:] = -kappa
    return K


def rotate(h, B, U):
    """(U^T h U, U^T B^J U)."""
    h, B, U = cc.as_t(h), cc.as_t(B), cc.as_t(U)
    return U.T @ h @ U, torch.einsum("rp,Jrs,sq->Jpq", U, B, U)


def fock(h, B, o: int):
    """Closed-shell Fock matrix F_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)] (R1 reading)."""
    h, B = cc.as_t(h), cc.as_t(B)
    dk = torch.einsum("Jkk->J", B[:, :o, :o])
    return h + 2.0 * torch.einsum("Jpq,J->pq", B, dk) - torch.einsum("Jpk,Jkq->pq", B[:, :, :o], B[:, :o, :])


def fock_ov_rotated(kappa, h, B, o: int):
    """F'[i][a] of the integrals rotated by exp(K(kappa))."""
    n = h.shape[0]
    U = torch.linalg.matrix_exp(kappa_matrix(kappa, o, n))
    hr, Br = rotate(h, B, U)
    return fock(hr, Br, o)[:o, o:]


def hf_hessian(h, B, o: int):
    """A^HF[ia][jb] = dF'_ia / dkappa_jb at kappa = 0, by differentiating through exp(K)."""
    h, B = cc.as_t(h), cc.as_t(B)
    n = h.shape[0]
    v = n - o
    z = torch.zeros((o, v), dtype=F64)
    J = torch.autograd.functional.jacobian(lambda k: fock_ov_rotated(k, h, B, o), z)
    return J.reshape(o * v, o * v)


def scf(h, B, o: int, tol=1e-13, maxit=50):
    """Nearest Hartree-Fock orbitals: Newton on F'_ia(kappa) = 0 from kappa = 0.

    Returns (kappa, U, h', B')."""
    h, B = cc.as_t(h), cc.as_t(B)
    n = h.shape[0]
    v = n - o
    kappa = torch.zeros((o, v), dtype=F64)
    for _ in range(maxit):
        f = fock_ov_rotated(kappa, h, B, o)
        if float(f.abs().max()) < tol:
            U = torch.linalg.matrix_exp(kappa_matrix(kappa, o, n))
            hr, Br = rotate(h, B, U)
            return kappa, U, hr, Br
        J = torch.autograd.functional.jacobian(lambda k: fock_ov_rotated(k, h, B, o), kappa).reshape(o * v, o * v)
        kappa = kappa - torch.linalg.solve(J, f.reshape(-1)).reshape(o, v)
    raise RuntimeError("Hartree-Fock equations not converged")


def rotation_direction(o: int, n: int, i: int, a: int):
    """dK/dkappa_ia as a matrix."""
    k = torch.zeros((o, n - o), dtype=F64)
    k[i, a] = 1.0
    return kappa_matrix(k, o, n)


# ---------------------------------------------------------------------------
# the relaxed coupling
# ---------------------------------------------------------------------------

def condition_derivative(S: System, res, i: int, j: int, mult, dh, dB) -> float:
    """Derivative of the amplitude and excited-state conditions of the Lagrangian
    along a Hamiltonian direction (dh, dB), at fixed amplitudes and multipliers:
    zeta.Omega^x + g0 eta^x.R_j + gamma.(A^x R_j) (for j = 0 the first term only)."""
    g0, gam, zeta = mult
    t = res.t
    dh, dB = cc.as_t(dh), cc.as_t(dB)
    ox1, ox2, _ = cc.hamiltonian_derivative_residual(t.x1, t.x2, S.h, S.B, dh, dB, S.o, **S.kw)
    f = zeta.dot(Vec(ox1, ox2))
    if j > 0:
        Rj = S.right_state(res, j)
        x1, x2, xe = cc.hamiltonian_derivative_jacobian(t.x1, t.x2, Rj.vec.x1, Rj.vec.x2, S.h, S.B, dh, dB, S.o,
                                                        **S.kw)
        f += g0 * float(xe) + gam.dot(Vec(x1, x2))
    return float(f)


def transition_density(S: System, res, L: State, R: State):
    """D_pq = <psi^L| E_pq |psi^R> = <HF|(l0 + L) exp(-T) E_pq exp(T) (r0 + R)|HF>.

    D is the derivative of <psi^L|H|psi^R> with respect to h_pq at fixed states.
    Expanding exp(-T) H exp(T) (r0 + R)|HF> over the reference, singles and
    doubles gives, with Omega, A and eta functions of (h, B) at fixed t,
      <psi^L|H|psi^R> = E (l0 r0 + L.R) + l0 eta.R + L.(r0 Omega + A R) + w.Omega,
    where w_k = <L| tau_k R_1 |HF> (doubles of L against singles of R times a
    singles excitation) carries R's singles through one more excitation.
    """
    t = res.t
    o = S.o
    w = S.tau_expectation(State(0.0, L.vec), State(0.0, Vec(R.vec.x1, torch.zeros_like(R.vec.x2))))
    w = Vec(w.x1, torch.zeros_like(w.x2))

    def phi(h):
        om1, om2, e = cc.residual(t.x1, t.x2, h, S.B, o, **S.kw)
        ar1, ar2 = cc.jacobian_right(t.x1, t.x2, R.vec.x1, R.vec.x2, h, S.B, o, **S.kw)
        et1, et2 = cc.eta(t.x1, t.x2, h, S.B, o, **S.kw)
        val = e * (L.c0 * R.c0 + L.vec.dot(R.vec))
        val = val + L.c0 * cc.pdot(et1, et2, R.vec.x1, R.vec.x2)
        val = val + cc.pdot(L.vec.x1, L.vec.x2, R.c0 * om1 + ar1, R.c0 * om2 + ar2)
        val = val + cc.pdot(w.x1, w.x2, om1, om2)
        return val

    return torch.func.grad(phi)(S.h.clone())


def kappa_eta(S: System, res, i: int, j: int, mult=None, tol_lin=1e-10):
    """k-eta[i][a] (Eq. orbitalrelax): D_ai - D_ia of the (i, j) transition density plus the
    derivative of the conditions along each occupied-virtual rotation of the integrals."""
    o, n = S.o, S.n
    v = n - o
    mult = mult if mult is not None else S.coupling_multipliers(res, i, j, tol_lin)
    Li = S.left_state(res, i)
    Rj = S.right_state(res, j)
    D = transition_density(S, res, Li, Rj)
    ke = torch.zeros((o, v), dtype=F64)
    for ii in range(o):
        for a in range(v):
            K = rotation_direction(o, n, ii, a)
            dh = K.T @ S.h + S.h @ K
            dB = torch.einsum("rp,Jrq->Jpq", K, S.B) + torch.einsum("Jpr,rq->Jpq", S.B, K)
            ke[ii, a] = D[o + a, ii] - D[ii, o + a] + condition_derivative(S, res, i, j, mult, dh, dB)
    return ke


def relaxed_coupling(S: System, res, i: int, j: int, h1, B1, tol_lin=1e-10):
    """F_ij^x with orbital relaxation: the unrelaxed value plus kappa-bar_ai F^x_ai."""
    o = S.o
    mult = S.coupling_multipliers(res, i, j, tol_lin)
    f0 = condition_derivative(S, res, i, j, mult, h1, B1)
    ke = kappa_eta(S, res, i, j, mult)
    A = hf_hessian(S.h, S.B, o)
    kbar = -torch.linalg.solve(A.T, ke.reshape(-1))
    h1, B1 = cc.as_t(h1), cc.as_t(B1)
    _, fx = torch.func.jvp(lambda hh, BB: fock(hh, BB, o)[:o, o:], (S.h, S.B), (h1, B1))
    return f0 + float(kbar @ fx.reshape(-1)), kbar.reshape(ke.shape)


def _rotation_integrals(S: System, ii: int, a: int):
    """(dh, dB) of the integrals along the rotation kappa_ia at kappa = 0."""
    K = rotation_direction(S.o, S.n, ii, a)
    dh = K.T @ S.h + S.h @ K
    dB = torch.einsum("rp,Jrq->Jpq", K, S.B) + torch.einsum("Jpr,rq->Jpq", S.B, K)
    return dh, dB


def relaxed_energy_gradient(S: System, res, k: int, h1, B1, tol_lin=1e-10):
    """dE_k/dx with the Hartree-Fock orbitals following x: the energy Lagrangian gains
    kappa-bar.F_ov with kappa-bar^T A^HF = -(k-eta_E)^T, k-eta_E the derivative of the energy
    Lagrangian along each occupied-virtual rotation of the integrals (no overlap term)."""
    o, v = S.o, S.n - S.o
    zeta = S.energy_multiplier(res, k, tol_lin)
    g0 = S.energy_lagrangian_derivative(res, k, zeta, h1, B1)
    ke = torch.zeros((o, v), dtype=F64)
    for ii in range(o):
        for a in range(v):
            ke[ii, a] = S.energy_lagrangian_derivative(res, k, zeta, *_rotation_integrals(S, ii, a))
    A = hf_hessian(S.h, S.B, o)
    kbar = -torch.linalg.solve(A.T, ke.reshape(-1))
    h1, B1 = cc.as_t(h1), cc.as_t(B1)
    _, fx = torch.func.jvp(lambda hh, BB: fock(hh, BB, o)[:o, o:], (S.h, S.B), (h1, B1))
    return g0 + float(kbar @ fx.reshape(-1))


def relaxed_energy_fd(h0, B0, h1, B1, o: int, k: int, nroots: int, delta=2e-3):
    """dE_k/dx by central differences (one Richardson step) with the Hartree-Fock orbitals
    re-optimised at every displacement; the root is followed by |L_k(x0).R(x)| (amplitudes in
    the rotated orbitals, a small rotation).  (h0, B0) must be Hartree-Fock at x0."""
    h0, B0, h1, B1 = (np.asarray(a, dtype=np.float64) for a in (h0, B0, h1, B1))
    eps = np.diag(np.asarray(fock(h0, B0, o)))
    S0 = System(eps, h0, B0, o)
    res0 = S0.run(nroots, dense=True, tol=1e-13, tol_lin=1e-13)

    def energy(x):
        _, _, hr, Br = scf(h0 + x * h1, B0 + x * B1, o)
        Sx = System(eps, hr, Br, o)
        tx, ex, _ = Sx.solve_ground(tol=1e-13, t0=res0.t)
        if k == 0:
            return float(ex)
        omega, R, _ = Sx.eom_dense(tx, nroots + 2)
        Lk = res0.left[k - 1].vec
        j = int(np.argmax([abs(Lk.dot(r)) for r in R]))
        return float(ex) + float(omega[j])

    E = {s: energy(s * delta) for s in (-2, -1, 1, 2)}
    return (8.0 * (E[1] - E[-1]) - (E[2] - E[-2])) / (12.0 * delta), S0, res0


# ---------------------------------------------------------------------------
# finite differences of the definition in determinant space (tiny systems)
# ---------------------------------------------------------------------------

def relaxed_overlap_fd(h0, B0, h1, B1, o: int, i: int, j: int, nroots: int, delta=2e-3):
    """d/dx <psi_i^L(x0)| psi_j^R(x)> by central differences (one Richardson step),
    with psi_j^R(x) computed in the Hartree-Fock orbitals at x and mapped to the x0
    orbitals by the rotation operator; (h0, B0) must be Hartree-Fock at x0.  The
    right state is normalised by L_j(x0)^T R_j(x) = 1 in amplitude space."""
    from .fockspace import CCBruteForce
    h0, B0, h1, B1 = (np.asarray(a, dtype=np.float64) for a in (h0, B0, h1, B1))
    n = h0.shape[0]
    eps = np.diag(np.asarray(fock(h0, B0, o)))
    S0 = System(eps, h0, B0, o)
    res0 = S0.run(nroots, dense=True, tol=1e-13, tol_lin=1e-13)
    bf0 = CCBruteForce(h0, B0, o)
    t0 = res0.t
    Li = S0.left_state(res0, i)
    bra = bf0.state_left(t0.x1.numpy(), t0.x2.numpy(), Li.c0, Li.vec.x1.numpy(), Li.vec.x2.numpy())
    fs = bf0.fs

    def overlap(x):
        hx, Bx = h0 + x * h1, B0 + x * B1
        kappa, U, hr, Br = scf(hx, Bx, o)
        Sx = System(eps, hr, Br, o)
        tx, _, _ = Sx.solve_ground(tol=1e-13, t0=t0)
        if j == 0:
            r0, rv = 1.0, Vec.zeros(o, n - o)
        else:
            omega, R, _ = Sx.eom_dense(tx, nroots + 2)
            Lj = res0.left[j - 1].vec
            k = int(np.argmax([abs(Lj.dot(r)) for r in R]))
            rv = R[k] / Lj.dot(R[k])
            r0 = float(Sx.eta(tx).dot(rv)) / omega[k]
        bfx = CCBruteForce(hr.numpy(), Br.numpy(), o)
        ket = bfx.state_right(tx.x1.numpy(), tx.x2.numpy(), r0, rv.x1.numpy(), rv.x2.numpy())
        K = kappa_matrix(kappa, o, n).numpy()
        X = sum(K[r, s] * fs.E(r, s) for r in range(n) for s in range(n) if K[r, s] != 0.0)
        return float(bra @ (scipy.linalg.expm(X) @ ket))

    O = {s: overlap(s * delta) for s in (-2, -1, 1, 2)}
    return (8.0 * (O[1] - O[-1]) - (O[2] - O[-2])) / (12.0 * delta), S0, res0
