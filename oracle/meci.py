"""Minimum-energy crossing point of two excited states along a synthetic family (test infrastructure).

The paper applies its couplings to locate conical intersections (Results section): the branching plane is
spanned by g = grad(E_2 - E_1) and h = (E_2 - E_1) F_12, and the search follows the Bearpark-Robb-Schlegel
direction G = P grad E_2 + 2 (E_2 - E_1) g/|g|, with P the projector onto the complement of the branching
plane.  The family here is synthetic: h(x) = h_0 + sum_a (x_a h_a + x_a^2 h_aa / 2), B(x) likewise, in a fixed
orthonormal orbital basis, so every derivative is a coupling or gradient along one direction
(dh/dx_a, dB/dx_a) at x.

Two sources of the state quantities are given: the CC oracle (energies, Lagrangian gradients, biorthonormal
couplings) and, for two electrons, full CI (Hellmann-Feynman gradients and the off-diagonal
Hellmann-Feynman coupling).  The biorthonormal F_12 differs from the FCI coupling by a positive state-scale
factor, which does not change the branching plane.
"""
from __future__ import annotations

import numpy as np

from .fockspace import CCBruteForce
from .solvers import System


class Family:
    """h(x) = h_0 + sum_a (x_a h_a + x_a^2/2 h_aa), B(x) likewise (quadratic terms optional)."""

    def __init__(self, eps, h0, B0, dirs, o: int, quad=None):
        self.eps, self.h0, self.B0, self.dirs, self.o = eps, np.asarray(h0), np.asarray(B0), dirs, o
        self.quad = quad if quad is not None else [(0.0 * dh, 0.0 * dB) for dh, dB in dirs]

    def hamiltonian(self, x):
        h = self.h0 + sum(xa * dh + 0.5 * xa * xa * qh for xa, (dh, _), (qh, _) in zip(x, self.dirs, self.quad))
        B = self.B0 + sum(xa * dB + 0.5 * xa * xa * qB for xa, (_, dB), (_, qB) in zip(x, self.dirs, self.quad))
        return h, B

    def directions(self, x):
        """(dh/dx_a, dB/dx_a) at x."""
        return [(dh + xa * qh, dB + xa * qB) for xa, (dh, dB), (qh, qB) in zip(x, self.dirs, self.quad)]


def cc_point(fam: Family, x, tol=1e-12):
    """(E_1, E_2, grad E_1, grad E_2, F_12 per direction) from the CC oracle at x."""
    h, B = fam.hamiltonian(x)
    S = System(fam.eps, h, B, fam.o)
    res = S.run(2, dense=True, tol=tol, tol_lin=tol)
    E = [res.e_ccsd + w for w in res.omega]
    dirs = fam.directions(x)
    g = [np.array([S.energy_gradient(res, k, dh, dB, tol_lin=tol) for dh, dB in dirs]) for k in (1, 2)]
    f12 = np.array([S.coupling(res, 1, 2, dh, dB, tol_lin=tol) for dh, dB in dirs])
    return E[0], E[1], g[0], g[1], f12


def fci_point(fam: Family, x):
    """The same quantities from full CI (exact for two electrons)."""
    h, B = fam.hamiltonian(x)
    bf = CCBruteForce(h, B, fam.o)
    w, U = bf.fci()
    Hx = [bf.hamiltonian_derivative(dh, B, dB) for dh, dB in fam.directions(x)]
    g = [np.array([U[:, k] @ Ha @ U[:, k] for Ha in Hx]) for k in (1, 2)]
    f12 = np.array([U[:, 1] @ Ha @ U[:, 2] / (w[2] - w[1]) for Ha in Hx])
    return w[1], w[2], g[0], g[1], f12


def bearpark_direction(E1, E2, g1, g2, f12):
    """G = P grad E_2 + 2 (E_2 - E_1) g/|g|, P projecting out span{g, h}, h = (E_2 - E_1) F_12."""
    g = g2 - g1
    q1 = g / np.linalg.norm(g)
    basis = [q1]
    hv = (E2 - E1) * f12
    hp = hv - (hv @ q1) * q1
    if np.linalg.norm(hp) > 1e-12 * max(np.linalg.norm(hv), 1e-300):
        basis.append(hp / np.linalg.norm(hp))
    P = np.eye(len(g)) - sum(np.outer(q, q) for q in basis)
    return P @ g2 + 2.0 * (E2 - E1) * q1


def search(point, x0, step=0.5, tol=1e-7, maxit=500):
    """x <- x - step G until |G| < tol; returns (x, number of steps, last point quantities)."""
    x = np.array(x0, dtype=float)
    for it in range(1, maxit + 1):
        q = point(x)
        G = bearpark_direction(*q)
        if np.linalg.norm(G) < tol:
            return x, it, q
        x = x - step * G
    raise RuntimeError("crossing search did not converge")
