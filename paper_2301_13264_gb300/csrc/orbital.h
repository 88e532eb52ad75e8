// Orbital relaxation: Hartree-Fock conditions and their derivatives as tensor programs.
//
// The Lagrangian of the Theory section holds the Hartree-Fock conditions F_ai = 0
// with multipliers kappa-bar (Eq. orbitalrelax): kappa-bar^T A^HF = -(k-eta)^T, and
// the coupling gains kappa-bar_ai F^q_ai (Eq. NAC_NC).  Orbitals rotate by
// U = exp(K) with occupied-virtual generators only, K[a][i] = kappa[i][a],
// K[i][a] = -kappa[i][a]; rotated integrals are h' = U^T h U, B'^J = U^T B^J U.
// Every quantity is a program over (h, B):
//   fock   F[i][a] = h_ia + sum_J [2 B^J_ia d_J - sum_k B^J_ik B^J_ka],  d_J = sum_k B^J_kk
//   rot    (dh, dB) = (K^T h + h K, K^T B^J + B^J K) for a direction x (all blocks)
//   hfA    A^HF x: the tangent of fock along rot(x)   (A^HF[ia][jb] = dF'_ia / dkappa_jb)
//   rotT   the adjoint of rot: (D, Z) -> x-bar, i.e. sum_pq D_pq dh_pq/dkappa + sum Z dB/dkappa
//   kdens  the adjoint of fock w.r.t. (h, B): densities of kappa-bar.F
//   rotate (h', B') = (U^T h U, U^T B U)
#pragma once

#include "ir.h"

namespace ccsd {

struct HFPrograms {
  Graph g;
  int h, B, ones_o;     // inputs (bound): integrals and a vector of o ones
  int U, hr, Br;        // rotate: U (bound) -> hr, Br (bound outputs)
  int F;                // fock output [o][v]
  int x, AX;            // hfA: direction x [o][v] -> A^HF x [o][v]
  int dD, dZ, xbar;     // rotT: seeds (D [n][n], Z [naux][n][n]) -> x-bar [o][v]
  int kbar, kH, kB;     // kdens: seed kappa-bar [o][v] -> (d/dh, d/dB) of kappa-bar.F
  Prog fock, hfA, rotT, kdens, rotate;
};

void build_hf_programs(HFPrograms& P);

}  // namespace ccsd
