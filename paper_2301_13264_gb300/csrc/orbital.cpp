// Orbital relaxation programs (see orbital.h).
#include "orbital.h"

namespace ccsd {

namespace {

struct Builder {
  Graph& g;
  Prog* p = nullptr;
  void C(Ref out, const char* lo, Ref a, const char* la, Ref b, const char* lb, double alpha) {
    Op op;
    op.kind = 'C';
    op.out = out;
    op.a = a;
    op.b = b;
    op.lo = lo;
    op.la = la;
    op.lb = lb;
    op.alpha = alpha;
    p->push_back(op);
  }
  void A(Ref out, const char* lo, Ref a, const char* la, double alpha) {
    Op op;
    op.kind = 'A';
    op.out = out;
    op.a = a;
    op.lo = lo;
    op.la = la;
    op.alpha = alpha;
    p->push_back(op);
  }
};

Prog concat(const Prog& a, const Prog& b) {
  Prog c = a;
  c.insert(c.end(), b.begin(), b.end());
  return c;
}

}  // namespace

void build_hf_programs(HFPrograms& P) {
  Graph& g = P.g;
  Builder bd{g};
  auto F = [&](int t) { return g.full(t); };
  auto V = [&](int t, const char* blk) { return g.view(t, blk); };

  P.h = g.add("h", "nn", ROLE_INPUT_H);
  P.B = g.add("B", "xnn", ROLE_INPUT_H);
  P.ones_o = g.add("ones_o", "o", ROLE_CONST);
  const int h = P.h, B = P.B;

  // fock: F[i][a] = h_ia + 2 sum_J B^J_ia d_J - sum_J sum_k B^J_ik B^J_ka
  Prog fock;
  bd.p = &fock;
  P.F = g.add("Fov", "ov", ROLE_OUTPUT);
  const int dJ = g.add("dJ", "x", ROLE_TEMP);
  bd.C(F(dJ), "P", V(B, "xoo"), "Pkk", F(P.ones_o), "k", 1.0);
  bd.A(F(P.F), "ia", V(h, "ov"), "ia", 1.0);
  bd.C(F(P.F), "ia", V(B, "xov"), "Pia", F(dJ), "P", 2.0);
  bd.C(F(P.F), "ia", V(B, "xoo"), "Pik", V(B, "xov"), "Pka", -1.0);
  P.fock = fock;

  // rot: (dh, dB) = (K^T h + h K, K^T B + B K) for the direction x (every block)
  Prog rot;
  bd.p = &rot;
  P.x = g.add("kx", "ov", ROLE_SEED);
  const int dh = g.add("rot_h", "nn", ROLE_TEMP);
  const int dB = g.add("rot_B", "xnn", ROLE_TEMP);
  const Ref x = F(P.x);
  // oo: sum_a x_ia M_aj + sum_a M_ia x_ja
  bd.C(V(dh, "oo"), "ij", x, "ia", V(h, "vo"), "aj", 1.0);
  bd.C(V(dh, "oo"), "ij", V(h, "ov"), "ia", x, "ja", 1.0);
  bd.C(V(dB, "xoo"), "Pij", x, "ia", V(B, "xvo"), "Paj", 1.0);
  bd.C(V(dB, "xoo"), "Pij", V(B, "xov"), "Pia", x, "ja", 1.0);
  // ov: sum_b x_ib M_ba - sum_j M_ij x_ja
  bd.C(V(dh, "ov"), "ia", x, "ib", V(h, "vv"), "ba", 1.0);
  bd.C(V(dh, "ov"), "ia", V(h, "oo"), "ij", x, "ja", -1.0);
  bd.C(V(dB, "xov"), "Pia", x, "ib", V(B, "xvv"), "Pba", 1.0);
  bd.C(V(dB, "xov"), "Pia", V(B, "xoo"), "Pij", x, "ja", -1.0);
  // vo: -sum_j x_ja M_ji + sum_b M_ab x_ib
  bd.C(V(dh, "vo"), "ai", x, "ja", V(h, "oo"), "ji", -1.0);
  bd.C(V(dh, "vo"), "ai", V(h, "vv"), "ab", x, "ib", 1.0);
  bd.C(V(dB, "xvo"), "Pai", x, "ja", V(B, "xoo"), "Pji", -1.0);
  bd.C(V(dB, "xvo"), "Pai", V(B, "xvv"), "Pab", x, "ib", 1.0);
  // vv: -sum_i x_ia M_ib - sum_i M_ai x_ib
  bd.C(V(dh, "vv"), "ab", x, "ia", V(h, "ov"), "ib", -1.0);
  bd.C(V(dh, "vv"), "ab", V(h, "vo"), "ai", x, "ib", -1.0);
  bd.C(V(dB, "xvv"), "Pab", x, "ia", V(B, "xov"), "Pib", -1.0);
  bd.C(V(dB, "xvv"), "Pab", V(B, "xvo"), "Pai", x, "ib", -1.0);

  // hfA: tangent of fock along rot(x)
  {
    std::map<int, int> tan = {{h, dh}, {B, dB}};
    Prog j = jvp(g, fock, tan, false, "HA");
    P.AX = tan.at(P.F);
    g.T[P.AX].role = ROLE_OUTPUT;
    P.hfA = concat(fock, concat(rot, j));
  }
  // rotT: adjoint of rot w.r.t. x
  {
    P.dD = g.add("rotT_D", "nn", ROLE_SEED);
    P.dZ = g.add("rotT_Z", "xnn", ROLE_SEED);
    std::map<int, int> adj = {{dh, P.dD}, {dB, P.dZ}};
    std::set<int> need = dependents(g, rot, {P.x});
    need.insert(P.x);
    P.rotT = vjp(g, rot, adj, need, false, "RT");
    P.xbar = adj.at(P.x);
    g.T[P.xbar].role = ROLE_OUTPUT;
  }
  // kdens: adjoint of fock w.r.t. (h, B) with seed kappa-bar on F
  {
    P.kbar = g.add("kbar", "ov", ROLE_SEED);
    std::map<int, int> adj = {{P.F, P.kbar}};
    std::set<int> need = dependents(g, fock, {h, B});
    need.insert(h);
    need.insert(B);
    Prog v = vjp(g, fock, adj, need, false, "KD");
    P.kdens = concat(fock, v);
    P.kH = adj.at(h);
    P.kB = adj.at(B);
    g.T[P.kH].role = g.T[P.kB].role = ROLE_OUTPUT;
  }
  // rotate: (U^T h U, U^T B U)
  {
    Prog r;
    bd.p = &r;
    P.U = g.add("U", "nn", ROLE_INPUT_H);
    P.hr = g.add("h_rot", "nn", ROLE_OUTPUT);
    P.Br = g.add("B_rot", "xnn", ROLE_OUTPUT);
    const int h1 = g.add("hU", "nn", ROLE_TEMP);
    const int B1 = g.add("BU", "xnn", ROLE_TEMP);
    bd.C(F(h1), "rq", F(h), "rs", F(P.U), "sq", 1.0);
    bd.C(F(P.hr), "pq", F(P.U), "rp", F(h1), "rq", 1.0);
    bd.C(F(B1), "Prq", F(B), "Prs", F(P.U), "sq", 1.0);
    bd.C(F(P.Br), "Ppq", F(P.U), "rp", F(B1), "Prq", 1.0);
    P.rotate = r;
  }
}

}  // namespace ccsd
