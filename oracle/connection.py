"""Orbital connections: the overlap term of the coupling (test infrastructure of the oracle).

The paper (section "Significance of orbital connections") writes the Hamiltonian, at every x, in
an orthonormal MO basis psi = T phi obtained from unmodified MOs phi(x) that are orthonormal only
at x0 (overlap S(x)).  The coupling then gains the derivative of the overlap of the two states'
orbital bases,

    O^q_ij = sum_rs D^ij_rs Y^q_rs,    Y^q_rs = <psi_r | d psi_s / dx_q> at x0,

with D^ij the transition density <psi_i^L| E_rs |psi_j^R>.  The natural connection has Y = 0, so
Eq. NAC_NC is complete; the symmetric connection T = S^(-1/2) has Y = (W - W^T)/2 with
W_rs = <phi_r | d phi_s / dx> the ket derivative of the unmodified MOs, so that
O^q_ij = sum_rs (D_rs - D_sr)/2 W_rs must be added.

Synthetic model (no atomic basis is involved): the unmodified-MO integrals h^U(x) = h0 + x h1,
B^U(x) = B0 + x B1 and a ket-derivative matrix W are given; to first order in x the unmodified MOs
have the overlap S(x) = 1 + x (W + W^T) among themselves and <phi(x0)|phi(x)> = 1 + x W with the
x0 ones.  The symmetric-connection integrals are h^sym(x) = T h^U(x) T and B^sym_J(x) = T B^U_J(x) T
with T = S(x)^(-1/2), so that along x
    dh^sym = h1 - (S1 h0 + h0 S1)/2,  dB^sym_J = B1_J - (S1 B0_J + B0_J S1)/2,  S1 = W + W^T.
Only first derivatives at x0 are used, so the model's second-order terms do not matter.

The finite-difference evaluation of the definition (determinant space, tiny systems) builds the
right state at x from (h^sym(x), B^sym(x)) in the basis psi(x) and maps it into the Fock space of
the x0 orbitals with the many-body operator of the one-particle overlap
U_rs = <psi_r(x0)|psi_s(x)> = sum_q <phi_r(x0)|phi_q(x)> T_qs(x).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import torch

from . import ccsd as cc
from .relaxed import transition_density
from .solvers import System, Vec

F64 = torch.float64


def symmetric_connection_derivatives(h0, B0, h1, B1, W):
    """(dh^sym, dB^sym): the x-derivative of the symmetric-connection integrals at x0."""
    h0, B0, h1, B1, W = (cc.as_t(a) for a in (h0, B0, h1, B1, W))
    S1 = W + W.T
    dh = h1 - 0.5 * (S1 @ h0 + h0 @ S1)
    dB = B1 - 0.5 * (torch.einsum("pr,Jrq->Jpq", S1, B0) + torch.einsum("Jpr,rq->Jpq", B0, S1))
    return dh, dB


def connection_term(S: System, res, i: int, j: int, W) -> float:
    """O_ij = sum_rs (D_rs - D_sr)/2 W_rs with D the (i, j) transition density at x0."""
    D = transition_density(S, res, S.left_state(res, i), S.right_state(res, j))
    W = cc.as_t(W)
    return float((0.5 * (D - D.T) * W).sum())


def symmetric_connection_coupling(S: System, res, i: int, j: int, h1, B1, W, tol_lin=1e-10) -> float:
    """F_ij along x in the symmetric connection: Eq. NAC_NC with the symmetric-connection
    Hamiltonian derivative, plus the overlap term O_ij."""
    dh, dB = symmetric_connection_derivatives(S.h, S.B, h1, B1, W)
    return S.coupling(res, i, j, dh, dB, tol_lin=tol_lin) + connection_term(S, res, i, j, W)


def symmetric_connection_fd(eps, h0, B0, h1, B1, W, o: int, i: int, j: int, nroots: int, delta=2e-3):
    """d/dx <psi_i^L(x0)|psi_j^R(x)> by central differences (one Richardson step) in determinant
    space, with the states at x built in the symmetric-connection basis and the ket carried into
    the x0 orbitals by the many-body operator of their one-particle overlap.  The right state is
    normalised by L_j(x0)^T R_j(x) = 1 in amplitude space, as in the natural-connection case."""
    from .fockspace import CCBruteForce
    h0, B0, h1, B1, W = (np.asarray(a, dtype=np.float64) for a in (h0, B0, h1, B1, W))
    n = h0.shape[0]
    S0 = System(eps, h0, B0, o)
    res0 = S0.run(nroots, dense=True, tol=1e-13, tol_lin=1e-13)
    bf0 = CCBruteForce(h0, B0, o)
    t0 = res0.t
    Li = S0.left_state(res0, i)
    bra = bf0.state_left(t0.x1.numpy(), t0.x2.numpy(), Li.c0, Li.vec.x1.numpy(), Li.vec.x2.numpy())
    fs = bf0.fs
    eye = np.eye(n)

    def overlap(x):
        Sx = eye + x * (W + W.T)
        w, V = np.linalg.eigh(Sx)
        T = (V / np.sqrt(w)) @ V.T  # S^(-1/2), symmetric
        hx = T @ (h0 + x * h1) @ T
        Bx = np.einsum("pr,Jrs,sq->Jpq", T, B0 + x * B1, T)
        Sys = System(eps, hx, Bx, o)
        tx, _, _ = Sys.solve_ground(tol=1e-13, t0=t0)
        if j == 0:
            r0, rv = 1.0, Vec.zeros(o, n - o)
        else:
            omega, R, _ = Sys.eom_dense(tx, nroots + 2)
            Lj = res0.left[j - 1].vec
            k = int(np.argmax([abs(Lj.dot(r)) for r in R]))
            rv = R[k] / Lj.dot(R[k])
            r0 = float(Sys.eta(tx).dot(rv)) / omega[k]
        ket = CCBruteForce(hx, Bx, o).state_right(tx.x1.numpy(), tx.x2.numpy(), r0, rv.x1.numpy(), rv.x2.numpy())
        U = (eye + x * W) @ T  # <psi_r(x0)|psi_s(x)>
        X = np.real(scipy.linalg.logm(U))
        G = sum(X[r, s] * fs.E(r, s) for r in range(n) for s in range(n) if X[r, s] != 0.0)
        return float(bra @ (scipy.linalg.expm(G) @ ket))

    O = {s: overlap(s * delta) for s in (-2, -1, 1, 2)}
    return (8.0 * (O[1] - O[-1]) - (O[2] - O[-2])) / (12.0 * delta), S0, res0
