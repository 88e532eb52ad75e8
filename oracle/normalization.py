"""Normalised-state couplings (test infrastructure of the oracle).

The paper compares its couplings with full CI, where states are normalised, through the
normalisation factor N^L of the left states (Implementation; Numerical examples, the LiH
comparison): with biorthonormal states N^R is approximately 1/N^L, and the normalised,
antisymmetrised coupling is

    Fbar_ij = ( N_i^L / N_j^L F_ij - N_j^L / N_i^L F_ji ) / 2.

N^L = 1/|psi^L| with <psi^L| = <HF|(l0 + L) exp(-T).  Because <mu|exp(-T) only de-excites, the
left state has no component beyond the doubles, so its norm is a finite sum: with
a_0 = <psi^L|HF> and a_mu = <psi^L|tau_mu|HF> (the packed manifold of the closed-shell
excitations),

    |psi^L|^2 = a_0^2 + sum_{mu,nu} a_mu a_nu <mu~|nu~>,

and the metric of the biorthonormal bras is 1/2 on the singles and, on the doubles stored
pair-symmetrically as A[i,j,a,b],

    sum_ijab (2 A_ijab^2 + A_ijab A_ijba) / 12 + (3/4) sum_ia A_iiaa^2.

(Read off the determinant space and pinned there.)  a_0 = l0 - L.t + L.(t1 t1) in the packed
inner product, a_mu = <L|tau_mu (1 - T_1)|HF>.
"""
from __future__ import annotations

import torch

from . import ccsd as cc
from .solvers import State, System, Vec

F64 = torch.float64


def left_components(S: System, res, k: int):
    """(a_0, a) of the left state k: a_0 = <psi_k^L|HF>, a = <psi_k^L|tau_mu|HF> (unpacked storage)."""
    L = S.left_state(res, k)
    t = res.t
    a0 = float(S.overlap(L, State(1.0, Vec.zeros(S.o, S.v)), t * -1.0))
    a = S.tau_expectation(L, State(1.0, Vec(-t.x1, torch.zeros_like(t.x2))))
    return a0, a


def bra_metric_norm2(a0: float, a: Vec) -> float:
    """a_0^2 + the biorthonormal-bra metric applied to (a_1, a_2)."""
    A = a.x2
    o, v = a.x1.shape
    q2 = (2.0 * A * A + A * A.permute(0, 1, 3, 2)).sum() / 12.0
    ii, aa = torch.meshgrid(torch.arange(o), torch.arange(v), indexing="ij")
    q2 = q2 + 0.75 * (A[ii, ii, aa, aa] ** 2).sum()
    return float(a0 * a0 + 0.5 * (a.x1 * a.x1).sum() + q2)


def left_norm(S: System, res, k: int) -> float:
    """N_k^L = 1/|psi_k^L| (k = 0: the ground state's left state <HF|(1 + Lambda) exp(-T))."""
    a0, a = left_components(S, res, k)
    return bra_metric_norm2(a0, a) ** -0.5


def normalized_coupling(S: System, res, i: int, j: int, h1, B1, tol_lin=1e-10) -> float:
    """(N_i^L / N_j^L F_ij - N_j^L / N_i^L F_ji) / 2 along (h1, B1)."""
    ni, nj = left_norm(S, res, i), left_norm(S, res, j)
    fij = S.coupling(res, i, j, h1, B1, tol_lin=tol_lin)
    fji = S.coupling(res, j, i, h1, B1, tol_lin=tol_lin)
    return 0.5 * (ni / nj * fij - nj / ni * fji)
