// The programs the coupling method runs, all derived from one residual program.
#pragma once

#include "ir.h"

namespace ccsd {

struct Programs {
  CCSDProgram cp;
  // residual: fwd_const once per Hamiltonian, fwd_t per amplitude vector
  // right transforms A R for a block of nvec vectors (seeds zR1/zR2 -> zAR1/zAR2/zAE)
  Prog jvp_z;
  int zR1, zR2, zAR1, zAR2, zAE;
  // left transforms (L^T A) and eta: seeds zL1/zL2/zLE on (O1,O2,E) -> zLA1/zLA2
  Prog vjp_z;
  int zL1, zL2, zLE, zLA1, zLA2;
  // second derivative: seeds (g1,g2,g0) on (O1,O2,E) and direction (r1,r2) ->
  // sum_nu d^2(g0 E + g.Omega)/dt dt_nu r_nu  (hF1, hF2)
  Prog hvp;
  int hG1, hG2, hG0, hR1, hR2, hF1, hF2;
  // densities: d/d(h,B) of z.Omega + g0 (eta.r) + g.(A r)  at fixed t
  Prog dens1;
  int dZ1, dZ2, dR1, dR2, dG1, dG2, dG0, dH, dB;
  // densities of z.Omega + e E at fixed t (right ground state; e E adds the energy's own density)
  Prog dens0;
  int eZ1, eZ2, eE, eH, eB;
};

void build_programs(Programs& P);

}  // namespace ccsd
