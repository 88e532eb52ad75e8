#include "programs.h"

#include <stdexcept>

namespace ccsd {

static Prog concat(const Prog& a, const Prog& b) {
  Prog c = a;
  c.insert(c.end(), b.begin(), b.end());
  return c;
}

void build_programs(Programs& P) {
  CCSDProgram& cp = P.cp;
  build_ccsd(cp);
  Graph& g = cp.g;
  const std::set<int> need_t = dependents(g, cp.fwd, {cp.t1, cp.t2});

  // A R: forward-mode tangents along a block of directions
  {
    P.zR1 = g.add("zR1", "zov", ROLE_SEED);
    P.zR2 = g.add("zR2", "zoovv", ROLE_SEED);
    std::map<int, int> tan = {{cp.t1, P.zR1}, {cp.t2, P.zR2}};
    P.jvp_z = jvp(g, cp.fwd, tan, true, "Jz");
    P.zAR1 = tan.at(cp.O1);
    P.zAR2 = tan.at(cp.O2);
    P.zAE = tan.at(cp.E);
    g.T[P.zAR1].role = g.T[P.zAR2].role = g.T[P.zAE].role = ROLE_OUTPUT;
  }
  // L^T A and eta: reverse mode
  {
    P.zL1 = g.add("zL1", "zov", ROLE_SEED);
    P.zL2 = g.add("zL2", "zoovv", ROLE_SEED);
    P.zLE = g.add("zLE", "z", ROLE_SEED);
    std::map<int, int> adj = {{cp.O1, P.zL1}, {cp.O2, P.zL2}, {cp.E, P.zLE}};
    P.vjp_z = vjp(g, cp.fwd, adj, need_t, true, "Vz");
    P.zLA1 = adj.at(cp.t1);
    P.zLA2 = adj.at(cp.t2);
    g.T[P.zLA1].role = g.T[P.zLA2].role = ROLE_OUTPUT;
  }
  // F-matrix (with energy part): tangent of the adjoint program
  {
    P.hG1 = g.add("hG1", "ov", ROLE_SEED);
    P.hG2 = g.add("hG2", "oovv", ROLE_SEED);
    P.hG0 = g.add("hG0", "", ROLE_SEED);
    std::map<int, int> adj = {{cp.O1, P.hG1}, {cp.O2, P.hG2}, {cp.E, P.hG0}};
    Prog v1 = vjp(g, cp.fwd, adj, need_t, false, "V1");
    P.hR1 = g.add("hR1", "ov", ROLE_SEED);
    P.hR2 = g.add("hR2", "oovv", ROLE_SEED);
    std::map<int, int> tan = {{cp.t1, P.hR1}, {cp.t2, P.hR2}};
    Prog j = jvp(g, concat(cp.fwd, v1), tan, false, "H1");
    P.hvp = concat(v1, j);
    P.hF1 = tan.at(adj.at(cp.t1));
    P.hF2 = tan.at(adj.at(cp.t2));
    g.T[P.hF1].role = g.T[P.hF2].role = ROLE_OUTPUT;
  }
  // densities with the excited right state
  {
    P.dR1 = g.add("dR1", "ov", ROLE_SEED);
    P.dR2 = g.add("dR2", "oovv", ROLE_SEED);
    std::map<int, int> tan = {{cp.t1, P.dR1}, {cp.t2, P.dR2}};
    Prog j = jvp(g, cp.fwd, tan, false, "JD");
    Prog pj = concat(cp.fwd, j);
    std::set<int> need_h = dependents(g, pj, {cp.h, cp.B});
    P.dZ1 = g.add("dZ1", "ov", ROLE_SEED);
    P.dZ2 = g.add("dZ2", "oovv", ROLE_SEED);
    P.dG1 = g.add("dG1", "ov", ROLE_SEED);
    P.dG2 = g.add("dG2", "oovv", ROLE_SEED);
    P.dG0 = g.add("dG0", "", ROLE_SEED);
    std::map<int, int> adj = {{cp.O1, P.dZ1}, {cp.O2, P.dZ2},
                              {tan.at(cp.O1), P.dG1}, {tan.at(cp.O2), P.dG2}, {tan.at(cp.E), P.dG0}};
    Prog v = vjp(g, pj, adj, need_h, false, "VD");
    P.dens1 = concat(j, v);
    P.dH = adj.at(cp.h);
    P.dB = adj.at(cp.B);
    g.T[P.dH].role = g.T[P.dB].role = ROLE_OUTPUT;
  }
  // densities with the ground right state: d/d(h,B) of z.Omega + e E
  {
    std::set<int> need_h = dependents(g, cp.fwd, {cp.h, cp.B});
    P.eZ1 = g.add("eZ1", "ov", ROLE_SEED);
    P.eZ2 = g.add("eZ2", "oovv", ROLE_SEED);
    P.eE = g.add("eE", "", ROLE_SEED);
    std::map<int, int> adj = {{cp.O1, P.eZ1}, {cp.O2, P.eZ2}, {cp.E, P.eE}};
    P.dens0 = vjp(g, cp.fwd, adj, need_h, false, "VE");
    P.eH = adj.at(cp.h);
    P.eB = adj.at(cp.B);
    g.T[P.eH].role = g.T[P.eB].role = ROLE_OUTPUT;
  }
}

}  // namespace ccsd
