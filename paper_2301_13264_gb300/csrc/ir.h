// Tensor-program IR for the closed-shell CCSD residual and its derivatives.
//
// The residual Omega(t; h, B) and energy E(t; h, B) (Theory section of the
// paper: Hbar = exp(-T) H exp(T) projected on the biorthonormal manifold) are
// written once as a list of tensor contractions.  Every quantity the coupling
// method needs is a derivative of that list:
//   A R          = forward-mode tangent along R             (Eq. for A)
//   L^T A, eta   = reverse-mode adjoint                     (Eq. for A, Lambda)
//   F(g) R       = tangent of the adjoint program           (Eq. for F)
//   densities    = adjoint w.r.t. (h, B) of zeta.Omega + g.(A R)  (Eq. NAC_NC)
// Each op is linear in each operand, so the derivative programs are again
// lists of contractions and permuted additions.
#pragma once

#include <cstdint>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace ccsd {

// Index classes of tensor dimensions:
//   'o' occupied (o), 'v' virtual (v), 'n' all orbitals (o+v),
//   'x' Cholesky index (naux), 'z' vector index of a block of trial vectors.
// A dimension of class 'n' can be viewed as its 'o' block [0,o) or 'v' block [o,n).
enum Role : int {
  ROLE_INPUT_T = 0,   // amplitudes (bound to caller or solver buffers)
  ROLE_INPUT_H = 1,   // Hamiltonian (h, B), owned by the handle
  ROLE_CONST = 2,     // identity / ones, filled at set-up
  ROLE_TEMP = 3,      // intermediate
  ROLE_OUTPUT = 4,    // program output (bound)
  ROLE_SEED = 5,      // tangent or adjoint seed (bound)
};

struct TensorInfo {
  std::string name;
  std::string cls;   // one class char per dimension; a leading 'z' marks a vector block
  int role = ROLE_TEMP;
};

struct Ref {
  int t = -1;
  std::string blk;   // per dimension: 'o'/'v'/'n' for class-n dims, else the class char
};

struct Op {
  char kind = 'C';   // 'C': out += alpha * sum a*b ; 'A': out += alpha * a (permuted)
  Ref out, a, b;
  std::string lo, la, lb;  // index labels per operand (repeated labels = diagonal)
  double alpha = 1.0;
};

using Prog = std::vector<Op>;

struct Graph {
  std::vector<TensorInfo> T;
  std::map<std::string, int> by_name;

  int add(const std::string& name, const std::string& cls, int role);
  int id(const std::string& name) const;
  Ref full(int t) const { return Ref{t, T[t].cls}; }
  Ref view(int t, const std::string& blk) const { return Ref{t, blk}; }
};

// Tensors that (transitively) depend on any tensor in `seeds` through `p`.
std::set<int> dependents(const Graph& g, const Prog& p, const std::set<int>& seeds);

// Forward-mode transform.  `tan` maps primal tensor -> tangent tensor for the
// seeds on entry and is extended with every tangent created.  With vec = true
// the tangents carry a leading 'z' dimension (a block of directions).
Prog jvp(Graph& g, const Prog& p, std::map<int, int>& tan, bool vec, const std::string& tag);

// Reverse-mode transform.  `adj` maps tensor -> adjoint tensor for the seeded
// outputs and is extended; only tensors in `need` receive adjoints.
Prog vjp(Graph& g, const Prog& p, std::map<int, int>& adj, const std::set<int>& need, bool vec,
         const std::string& tag);

// Text form of a program (tensors + ops), used by the host-side tests.
std::string dump(const Graph& g, const Prog& p);

// Residual program builder: returns the forward program and the names of its
// inputs/outputs.  Tensors: t1[o,v] t2[o,o,v,v] h[n,n] B[x,n,n] ->
// O1[o,v] O2[o,o,v,v] E[] (scalar).
struct CCSDProgram {
  Graph g;
  Prog fwd;           // whole forward program
  Prog fwd_const;     // ops depending only on (h, B)
  Prog fwd_t;         // ops depending on t
  int t1, t2, h, B, O1, O2, E, eye, ones_o;
};
void build_ccsd(CCSDProgram& cp);

}  // namespace ccsd
