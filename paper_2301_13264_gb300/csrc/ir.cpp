// Tensor-program IR: graph bookkeeping, derivative transforms, the CCSD
// residual program.  Host-only code.
#include "ir.h"

#include <algorithm>
#include <sstream>
#include <stdexcept>

namespace ccsd {

int Graph::add(const std::string& name, const std::string& cls, int role) {
  if (by_name.count(name)) throw std::runtime_error("duplicate tensor " + name);
  T.push_back(TensorInfo{name, cls, role});
  int id = (int)T.size() - 1;
  by_name[name] = id;
  return id;
}

int Graph::id(const std::string& name) const {
  auto it = by_name.find(name);
  if (it == by_name.end()) throw std::runtime_error("no tensor " + name);
  return it->second;
}

std::set<int> dependents(const Graph& g, const Prog& p, const std::set<int>& seeds) {
  (void)g;
  std::set<int> dep = seeds;
  bool changed = true;
  while (changed) {  // programs may write a tensor in several ops; iterate to a fixed point
    changed = false;
    for (const Op& op : p) {
      bool d = dep.count(op.a.t) || (op.kind == 'C' && dep.count(op.b.t));
      if (d && !dep.count(op.out.t)) {
        dep.insert(op.out.t);
        changed = true;
      }
    }
  }
  return dep;
}

static Ref vref(const Ref& r, int t, bool vec) {
  Ref o;
  o.t = t;
  o.blk = vec ? "z" + r.blk : r.blk;
  return o;
}

static int derived(Graph& g, int t, bool vec, const std::string& tag, int role) {
  const TensorInfo& ti = g.T[t];
  std::string name = tag + "(" + ti.name + ")";
  auto it = g.by_name.find(name);
  if (it != g.by_name.end()) return it->second;
  std::string cls = vec ? "z" + ti.cls : ti.cls;
  return g.add(name, cls, role);
}

Prog jvp(Graph& g, const Prog& p, std::map<int, int>& tan, bool vec, const std::string& tag) {
  Prog out;
  const std::string z = vec ? "z" : "";
  for (const Op& op : p) {
    auto ta = tan.find(op.a.t);
    bool has_a = ta != tan.end();
    bool has_b = false;
    int tb = -1;
    if (op.kind == 'C') {
      auto it = tan.find(op.b.t);
      if (it != tan.end()) {
        has_b = true;
        tb = it->second;
      }
    }
    if (!has_a && !has_b) continue;
    int to;
    auto it = tan.find(op.out.t);
    if (it != tan.end()) {
      to = it->second;
    } else {
      to = derived(g, op.out.t, vec, tag, ROLE_TEMP);
      tan[op.out.t] = to;
    }
    if (op.kind == 'A') {
      Op n;
      n.kind = 'A';
      n.out = vref(op.out, to, vec);
      n.a = vref(op.a, ta->second, vec);
      n.lo = z + op.lo;
      n.la = z + op.la;
      n.alpha = op.alpha;
      out.push_back(n);
      continue;
    }
    if (has_a) {
      Op n = op;
      n.out = vref(op.out, to, vec);
      n.a = vref(op.a, ta->second, vec);
      n.lo = z + op.lo;
      n.la = z + op.la;
      out.push_back(n);
    }
    if (has_b) {
      Op n = op;
      n.out = vref(op.out, to, vec);
      n.b = vref(op.b, tb, vec);
      n.lo = z + op.lo;
      n.lb = z + op.lb;
      out.push_back(n);
    }
  }
  return out;
}

Prog vjp(Graph& g, const Prog& p, std::map<int, int>& adj, const std::set<int>& need, bool vec,
         const std::string& tag) {
  Prog out;
  const std::string z = vec ? "z" : "";
  auto adj_of = [&](int t) {
    auto it = adj.find(t);
    if (it != adj.end()) return it->second;
    int a = derived(g, t, vec, tag, ROLE_TEMP);
    adj[t] = a;
    return a;
  };
  for (auto rit = p.rbegin(); rit != p.rend(); ++rit) {
    const Op& op = *rit;
    auto ao = adj.find(op.out.t);
    if (ao == adj.end()) continue;
    Ref obar = vref(op.out, ao->second, vec);
    if (op.kind == 'A') {
      if (!need.count(op.a.t)) continue;
      Op n;
      n.kind = 'A';
      n.out = vref(op.a, adj_of(op.a.t), vec);
      n.lo = z + op.la;
      n.a = obar;
      n.la = z + op.lo;
      n.alpha = op.alpha;
      out.push_back(n);
      continue;
    }
    if (need.count(op.a.t)) {
      Op n;
      n.kind = 'C';
      n.out = vref(op.a, adj_of(op.a.t), vec);
      n.lo = z + op.la;
      n.a = obar;
      n.la = z + op.lo;
      n.b = op.b;
      n.lb = op.lb;
      n.alpha = op.alpha;
      out.push_back(n);
    }
    if (need.count(op.b.t)) {
      Op n;
      n.kind = 'C';
      n.out = vref(op.b, adj_of(op.b.t), vec);
      n.lo = z + op.lb;
      n.a = op.a;
      n.la = op.la;
      n.b = obar;
      n.lb = z + op.lo;
      n.alpha = op.alpha;
      out.push_back(n);
    }
  }
  return out;
}

std::string dump(const Graph& g, const Prog& p) {
  std::ostringstream s;
  s.precision(17);
  std::set<int> used;
  for (const Op& op : p) {
    used.insert(op.out.t);
    used.insert(op.a.t);
    if (op.kind == 'C') used.insert(op.b.t);
  }
  auto lab = [](const std::string& l) { return l.empty() ? std::string("-") : l; };
  for (int t : used) s << "T " << t << " " << g.T[t].name << " " << g.T[t].role << " " << lab(g.T[t].cls) << "\n";
  for (const Op& op : p) {
    if (op.kind == 'C')
      s << "C " << op.out.t << " " << lab(op.out.blk) << " " << lab(op.lo) << " " << op.a.t << " "
        << lab(op.a.blk) << " " << lab(op.la) << " " << op.b.t << " " << lab(op.b.blk) << " " << lab(op.lb) << " "
        << op.alpha << "\n";
    else
      s << "A " << op.out.t << " " << lab(op.out.blk) << " " << lab(op.lo) << " " << op.a.t << " " << lab(op.a.blk)
        << " " << lab(op.la) << " " << op.alpha << "\n";
  }
  return s.str();
}

// ---------------------------------------------------------------------------
// The closed-shell CCSD residual over Cholesky factors, T1-transformed.
//
// With t1 placed in the (virtual, occupied) block, exp(-T1) H exp(T1) has
// integrals h^ = (1 - t1) h (1 + t1) and B^ = (1 - t1) B (1 + t1); by blocks
//   B^_oo = B_oo + B_ov t1^T,  B^_ov = B_ov,  B^_vv = B_vv - t1^T B_ov,
//   B^_vo = B_vo + B_vv t1^T - t1^T B^_oo.
// The doubles terms over these integrals (u = 2 t_ij^ab - t_ij^ba, L = 2g - g'):
//   Omega_ai  = F_ai + u_ki^cd g_adkc - u_kl^ac g_kilc + u_ik^ac F_kc
//   Omega_aibj = P[ 1/2 g_aibj + 1/2 t_ij^cd g_acbd + 1/2 t_kl^ab (g_kilj + t_ij^cd g_kcld)
//     - 1/2 t_kj^bc C_kiac - t_ki^bc C_kjac + 1/2 u_jk^bc D_aikc
//     + t_ij^ac (F_bc - u_kl^bd g_ldkc) - t_ik^ab (F_kj + u_lj^cd g_kdlc) ]
//   C_kiac = g_kiac - 1/2 t_li^ad g_kdlc,  D_aikc = L_aikc + 1/2 u_il^ad L_ldkc
//   E = sum_i (h^_ii + F_ii) + t_ij^ab L_iajb,
// with P X_aibj = X_aibj + X_bjai.  The particle-particle ladder uses the dressed
// vvvv integrals; since B^_vv = B_vv - t1^T B_ov they expand into the bare
// W_abcd = (ac|bd) (built once) plus ovvv and ovov pieces:
//   t_ij^cd g^_acbd = t_ij^cd W_abcd - t_ak V_ijkb - t_bl V_jila + t_ak t_bl U_ijkl,
//   V_ijkb = t_ij^cd (kc|bd),  U_ijkl = t_ij^cd (kc|ld).
// ---------------------------------------------------------------------------
void build_ccsd(CCSDProgram& cp) {
  Graph& g = cp.g;
  Prog& p = cp.fwd;
  auto tmp = [&](const char* name, const char* cls) { return g.add(name, cls, ROLE_TEMP); };
  auto F = [&](int t) { return g.full(t); };
  auto Vw = [&](int t, const char* blk) { return g.view(t, blk); };
  auto Cn = [&](Ref out, const char* lo, Ref a, const char* la, Ref b, const char* lb, double alpha) {
    Op op;
    op.kind = 'C';
    op.out = out;
    op.a = a;
    op.b = b;
    op.lo = lo;
    op.la = la;
    op.lb = lb;
    op.alpha = alpha;
    p.push_back(op);
  };
  auto Ax = [&](Ref out, const char* lo, Ref a, const char* la, double alpha) {
    Op op;
    op.kind = 'A';
    op.out = out;
    op.a = a;
    op.lo = lo;
    op.la = la;
    op.alpha = alpha;
    p.push_back(op);
  };

  cp.t1 = g.add("t1", "ov", ROLE_INPUT_T);
  cp.t2 = g.add("t2", "oovv", ROLE_INPUT_T);
  cp.h = g.add("h", "nn", ROLE_INPUT_H);
  cp.B = g.add("B", "xnn", ROLE_INPUT_H);
  cp.ones_o = g.add("ones_o", "o", ROLE_CONST);
  cp.eye = -1;
  const int t1 = cp.t1, t2 = cp.t2, h = cp.h, B = cp.B, one = cp.ones_o;
  const Ref h_oo = Vw(h, "oo"), h_ov = Vw(h, "ov"), h_vo = Vw(h, "vo"), h_vv = Vw(h, "vv");
  const Ref B_oo = Vw(B, "xoo"), B_ov = Vw(B, "xov"), B_vo = Vw(B, "xvo"), B_vv = Vw(B, "xvv");

  // bare integral blocks (depend on B only; hoisted)
  int W = tmp("W", "vvvv");        // W[a,b,c,d] = (ac|bd)
  Cn(F(W), "abcd", B_vv, "Pac", B_vv, "Pbd", 1.0);
  int Gs = tmp("Govvv", "ovvv");   // Gs[k,b,c,d] = (kc|bd)
  Cn(F(Gs), "kbcd", B_ov, "Pkc", B_vv, "Pbd", 1.0);
  int Gov = tmp("Govov", "ovov");  // Gov[k,c,l,d] = (kc|ld)
  Cn(F(Gov), "kcld", B_ov, "Pkc", B_ov, "Pld", 1.0);
  int Lov = tmp("Lovov", "ovov");  // Lov[l,d,k,c] = 2 (ld|kc) - (lc|kd)
  Ax(F(Lov), "ldkc", F(Gov), "ldkc", 2.0);
  Ax(F(Lov), "ldkc", F(Gov), "lckd", -1.0);

  // T1-dressed one-electron integrals
  int hh_oo = tmp("hh_oo", "oo");
  Ax(F(hh_oo), "ij", h_oo, "ij", 1.0);
  Cn(F(hh_oo), "ij", h_ov, "ic", F(t1), "jc", 1.0);
  int hh_vv = tmp("hh_vv", "vv");
  Ax(F(hh_vv), "ab", h_vv, "ab", 1.0);
  Cn(F(hh_vv), "ab", F(t1), "ka", h_ov, "kb", -1.0);
  int hh_vo = tmp("hh_vo", "vo");
  Ax(F(hh_vo), "ai", h_vo, "ai", 1.0);
  Cn(F(hh_vo), "ai", h_vv, "ac", F(t1), "ic", 1.0);
  Cn(F(hh_vo), "ai", F(t1), "ka", F(hh_oo), "ki", -1.0);

  // T1-dressed Cholesky blocks
  int Bh_oo = tmp("Bh_oo", "xoo");
  Ax(F(Bh_oo), "Pij", B_oo, "Pij", 1.0);
  Cn(F(Bh_oo), "Pij", B_ov, "Pic", F(t1), "jc", 1.0);
  int Bh_vv = tmp("Bh_vv", "xvv");
  Ax(F(Bh_vv), "Pab", B_vv, "Pab", 1.0);
  Cn(F(Bh_vv), "Pab", F(t1), "ka", B_ov, "Pkb", -1.0);
  int Bh_vo = tmp("Bh_vo", "xvo");
  Ax(F(Bh_vo), "Pai", B_vo, "Pai", 1.0);
  Cn(F(Bh_vo), "Pai", B_vv, "Pac", F(t1), "ic", 1.0);
  Cn(F(Bh_vo), "Pai", F(t1), "ka", F(Bh_oo), "Pki", -1.0);

  // Fock matrix F_pq = h^_pq + 2 sum_P B^_pq d_P - sum_Pk B^_pk B^_kq, d_P = sum_k B^_kk
  int d = tmp("dP", "x");
  Cn(F(d), "P", F(Bh_oo), "Pkk", F(one), "k", 1.0);
  int F_oo = tmp("F_oo", "oo");
  Ax(F(F_oo), "kj", F(hh_oo), "kj", 1.0);
  Cn(F(F_oo), "kj", F(Bh_oo), "Pkj", F(d), "P", 2.0);
  Cn(F(F_oo), "kj", F(Bh_oo), "Pkl", F(Bh_oo), "Plj", -1.0);
  int F_ov = tmp("F_ov", "ov");
  Ax(F(F_ov), "kc", h_ov, "kc", 1.0);
  Cn(F(F_ov), "kc", B_ov, "Pkc", F(d), "P", 2.0);
  Cn(F(F_ov), "kc", F(Bh_oo), "Pkl", B_ov, "Plc", -1.0);
  int F_vo = tmp("F_vo", "vo");
  Ax(F(F_vo), "ai", F(hh_vo), "ai", 1.0);
  Cn(F(F_vo), "ai", F(Bh_vo), "Pai", F(d), "P", 2.0);
  Cn(F(F_vo), "ai", F(Bh_vo), "Pal", F(Bh_oo), "Pli", -1.0);
  int F_vv = tmp("F_vv", "vv");
  Ax(F(F_vv), "bc", F(hh_vv), "bc", 1.0);
  Cn(F(F_vv), "bc", F(Bh_vv), "Pbc", F(d), "P", 2.0);
  Cn(F(F_vv), "bc", F(Bh_vo), "Pbl", B_ov, "Plc", -1.0);

  // energy
  cp.E = g.add("E", "", ROLE_OUTPUT);
  Cn(F(cp.E), "", F(hh_oo), "ii", F(one), "i", 1.0);
  Cn(F(cp.E), "", F(F_oo), "ii", F(one), "i", 1.0);
  Cn(F(cp.E), "", F(t2), "ijab", F(Lov), "iajb", 1.0);

  int u = tmp("u", "oovv");
  Ax(F(u), "ijab", F(t2), "ijab", 2.0);
  Ax(F(u), "ijab", F(t2), "ijba", -1.0);

  // singles
  cp.O1 = g.add("O1", "ov", ROLE_OUTPUT);
  const int O1 = cp.O1;
  Ax(F(O1), "ia", F(F_vo), "ai", 1.0);
  int Yd = tmp("Yd", "xov");
  Cn(F(Yd), "Pid", F(u), "kicd", B_ov, "Pkc", 1.0);
  Cn(F(O1), "ia", F(Bh_vv), "Pad", F(Yd), "Pid", 1.0);
  Cn(F(O1), "ia", F(Bh_oo), "Pki", F(Yd), "Pka", -1.0);
  Cn(F(O1), "ia", F(u), "ikac", F(F_ov), "kc", 1.0);

  // doubles, before the pair permutation
  int Rd = tmp("Rd", "oovv");
  Cn(F(Rd), "ijab", F(Bh_vo), "Pai", F(Bh_vo), "Pbj", 0.5);
  Cn(F(Rd), "ijab", F(t2), "ijcd", F(W), "abcd", 0.5);
  int Vt = tmp("Vt", "ooov");
  Cn(F(Vt), "ijkb", F(t2), "ijcd", F(Gs), "kbcd", 1.0);
  Cn(F(Rd), "ijab", F(t1), "ka", F(Vt), "ijkb", -1.0);
  int U = tmp("U", "oooo");
  Cn(F(U), "ijkl", F(t2), "ijcd", F(Gov), "kcld", 1.0);
  int chi = tmp("chi", "oooo");
  Cn(F(chi), "kilj", F(Bh_oo), "Pki", F(Bh_oo), "Plj", 1.0);
  Ax(F(chi), "kilj", F(U), "ijkl", 1.0);
  Cn(F(Rd), "ijab", F(t2), "klab", F(chi), "kilj", 0.5);
  int S1 = tmp("S1", "oovo");
  Cn(F(S1), "ijal", F(t1), "ka", F(U), "ijkl", 1.0);
  Cn(F(Rd), "ijab", F(t1), "lb", F(S1), "ijal", 0.5);
  int Gk = tmp("Gk", "oovv");  // Gk[k,i,a,c] = (ki|ac)^
  Cn(F(Gk), "kiac", F(Bh_oo), "Pki", F(Bh_vv), "Pac", 1.0);
  int Cm = tmp("Cm", "oovv");
  Ax(F(Cm), "kiac", F(Gk), "kiac", 1.0);
  Cn(F(Cm), "kiac", F(t2), "liad", F(Gov), "kdlc", -0.5);
  Cn(F(Rd), "ijab", F(t2), "kjbc", F(Cm), "kiac", -0.5);
  Cn(F(Rd), "ijab", F(t2), "kibc", F(Cm), "kjac", -1.0);
  int Dm = tmp("Dm", "voov");
  Cn(F(Dm), "aikc", F(Bh_vo), "Pai", B_ov, "Pkc", 2.0);
  Ax(F(Dm), "aikc", F(Gk), "kiac", -1.0);
  Cn(F(Dm), "aikc", F(u), "ilad", F(Lov), "ldkc", 0.5);
  Cn(F(Rd), "ijab", F(u), "jkbc", F(Dm), "aikc", 0.5);
  int Gvv = tmp("Gvv", "vv");
  Ax(F(Gvv), "bc", F(F_vv), "bc", 1.0);
  Cn(F(Gvv), "bc", F(u), "klbd", F(Gov), "ldkc", -1.0);
  Cn(F(Rd), "ijab", F(t2), "ijac", F(Gvv), "bc", 1.0);
  int Goo = tmp("Goo", "oo");
  Ax(F(Goo), "kj", F(F_oo), "kj", 1.0);
  Cn(F(Goo), "kj", F(u), "ljcd", F(Gov), "kdlc", 1.0);
  Cn(F(Rd), "ijab", F(t2), "ikab", F(Goo), "kj", -1.0);

  cp.O2 = g.add("O2", "oovv", ROLE_OUTPUT);
  Ax(F(cp.O2), "ijab", F(Rd), "ijab", 1.0);
  Ax(F(cp.O2), "ijab", F(Rd), "jiba", 1.0);

  // split into Hamiltonian-only and t-dependent parts
  std::set<int> tdep = dependents(g, p, {t1, t2});
  for (const Op& op : p) {
    if (tdep.count(op.out.t))
      cp.fwd_t.push_back(op);
    else
      cp.fwd_const.push_back(op);
  }
}

}  // namespace ccsd
