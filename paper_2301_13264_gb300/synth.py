"""Seeded synthetic closed-shell Hamiltonians.

This module only draws random numbers; it holds none of the method's
arithmetic (no Fock build, no integrals, no amplitudes).  Both the CUDA path
and the CPU oracle consume what it returns.

Recipe (Theory section of the paper: a closed-shell Hamiltonian given by
one-electron integrals h_pq and Cholesky-factored two-electron integrals
g_pqrs = sum_J B^J_pq B^J_rs, with a perturbation direction x entering as
h(x) = h0 + x h1 and B(x) = B0 + x B1):

* orbital energies: eps_occ ~ U[-2.0, -0.3], eps_vir ~ U[0.1, 3.0], each sorted
  ascending; occupied orbitals come first.
* h0 = diag(eps) + a symmetric matrix whose strict upper triangle is drawn
  N(0, 0.05) and mirrored.  The reference determinant is therefore not a
  Hartree-Fock solution (F_ai != 0); T1 absorbs the orbital relaxation.
* B0^J symmetric in pq, upper triangle (diagonal included) ~ N(0, 0.1/sqrt(naux)).
* h1: symmetric, upper triangle (diagonal included) ~ 0.1 * N(0, 0.05).
* B1^J: symmetric, upper triangle ~ 0.1 * N(0, 0.1/sqrt(naux)).
* draw order from numpy.random.default_rng(seed): eps_occ, eps_vir, h noise,
  B0, h1, B1.
* optional virtual gap: eps_vir[1] = eps_vir[0] + gap and the rest shifted up
  so that eps_vir[2] >= eps_vir[1] + 0.5, which isolates two low roots.

"N(0, s)" means standard deviation s.  All arrays are float64, row-major:
eps[n], h[n, n], B[naux, n, n] with n = o + v.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Hamiltonian", "make_hamiltonian", "WORKLOADS", "workload", "random_amplitudes"]


@dataclass
class Hamiltonian:
    o: int
    v: int
    naux: int
    eps: np.ndarray   # [n]
    h: np.ndarray     # [n, n]
    B: np.ndarray     # [naux, n, n]
    h1: np.ndarray    # [n, n]      perturbation direction for h
    B1: np.ndarray    # [naux, n, n] perturbation direction for B
    seed: int

    @property
    def n(self) -> int:
        return self.o + self.v

    def at(self, x: float) -> "Hamiltonian":
        """The Hamiltonian displaced by x along (h1, B1)."""
        return Hamiltonian(self.o, self.v, self.naux, self.eps.copy(),
                           self.h + x * self.h1, self.B + x * self.B1,
                           self.h1, self.B1, self.seed)


def _sym_upper(rng: np.random.Generator, n: int, scale: float, diag: bool) -> np.ndarray:
    """Symmetric n x n matrix from an upper triangle of N(0, scale) draws."""
    k = 0 if diag else 1
    iu = np.triu_indices(n, k)
    m = np.zeros((n, n))
    m[iu] = rng.normal(0.0, scale, size=iu[0].size)
    return m + np.triu(m, 1).T


def _sym_upper_batch(rng: np.random.Generator, nb: int, n: int, scale: float) -> np.ndarray:
    iu = np.triu_indices(n, 0)
    out = np.zeros((nb, n, n))
    vals = rng.normal(0.0, scale, size=(nb, iu[0].size))
    out[:, iu[0], iu[1]] = vals
    out[:, iu[1], iu[0]] = vals
    return out


def make_hamiltonian(o: int, v: int, naux: int, seed: int = 0, vir_gap: float | None = None,
                     hnoise: float = 0.05, bscale: float = 0.1, pert: float = 0.1) -> Hamiltonian:
    if o < 1 or v < 1 or naux < 1:
        raise ValueError("o, v, naux must be positive")
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-2.0, -0.3, size=o))
    eps_v = np.sort(rng.uniform(0.1, 3.0, size=v))
    if vir_gap is not None and v >= 2:
        eps_v[1] = eps_v[0] + vir_gap
        if v >= 3:
            shift = max(0.0, eps_v[1] + 0.5 - eps_v[2])
            eps_v[2:] += shift
    eps = np.concatenate([eps_o, eps_v])
    n = o + v
    h = np.diag(eps) + _sym_upper(rng, n, hnoise, diag=False)
    bs = bscale / np.sqrt(naux)
    B = _sym_upper_batch(rng, naux, n, bs)
    h1 = pert * _sym_upper(rng, n, hnoise, diag=True)
    B1 = _sym_upper_batch(rng, naux, n, pert * bs)
    return Hamiltonian(o, v, naux, eps, h, B, h1, B1, seed)


# Named workloads.  The thymine shapes follow the molecule of the paper's last
# example (C5H6N2O2: 66 electrons, so 33 doubly occupied orbitals; 156 basis
# functions in cc-pVDZ and 261 in aug-cc-pVDZ), with naux about 3.5 n.
WORKLOADS = {
    "small": dict(o=5, v=20, naux=75, seed=0),
    "thymine_dz": dict(o=33, v=123, naux=550, seed=0, vir_gap=0.25),
    "thymine_adz": dict(o=33, v=228, naux=900, seed=0),
}


def workload(name: str) -> Hamiltonian:
    return make_hamiltonian(**WORKLOADS[name])


def random_amplitudes(o: int, v: int, seed: int, scale: float = 0.01, nvec: int = 1):
    """Seeded random singles/doubles vectors in the library's layout.

    Singles are [i][a]; doubles are [i][j][a][b] with x_ijab = x_jiba (the pair
    symmetry of closed-shell doubles).  Returns (x1[nvec,o,v], x2[nvec,o,o,v,v]).
    """
    rng = np.random.default_rng(seed)
    x1 = rng.normal(0.0, scale, size=(nvec, o, v))
    x2 = rng.normal(0.0, scale, size=(nvec, o, o, v, v))
    x2 = 0.5 * (x2 + x2.transpose(0, 2, 1, 4, 3))
    return x1, x2
