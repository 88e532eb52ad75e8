"""Literal determinant-space evaluation of the CC quantities (tiny systems only).

Test infrastructure of the oracle.  Nothing here uses the CCSD working
equations: every quantity is computed from its definition in the paper's
Theory section, with explicit matrices on the Sz = 0 determinant space of n
spatial orbitals and 2o electrons:

* H = sum_pq h_pq E_pq + 1/2 sum_pqrs g_pqrs (E_pq E_rs - delta_qr E_ps) with
  the singlet excitation operators E_pq = a+_pa a_qa + a+_pb a_qb;
* T = sum_mu t_mu tau_mu with tau_ai = E_ai and doubles T2 = 1/2 sum t_aibj E_ai E_bj;
* Hbar = exp(-T) H exp(T) (T is nilpotent, the series is summed exactly);
* the biorthonormal projection <mu~| defined by <mu~|tau_nu|HF> = delta_mu,nu on
  the packed manifold {tau_ai} U {tau_aibj, ai >= bj}, tau_aibj = E_ai E_bj for
  ai > bj and tau_aiai = E_ai E_ai / 2 (so T2 above equals sum_{ai>=bj} t tau);
* Omega_mu = <mu~|Hbar|HF>, E = <HF|Hbar|HF>, A_mu,nu = <mu~|[Hbar, tau_nu]|HF>,
  eta_nu = <HF|[Hbar, tau_nu]|HF>, F(g)_mu,nu = <g|[[Hbar, tau_mu], tau_nu]|HF>.

Vectors are exchanged with the closed-shell engine in its unpacked layout:
singles x1[i, a], doubles x2[i, j, a, b] with x2[i,j,a,b] = x2[j,i,b,a] equal to
the packed coefficient of tau_aibj.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _popcount(x: int) -> int:
    return bin(x).count("1")


class FockSpace:
    """Sz = 0 determinant space for n spatial orbitals, o doubly occupied in HF."""

    def __init__(self, n: int, o: int):
        self.n, self.o, self.v = n, o, n - o
        self.strings = [sum(1 << p for p in c) for c in itertools.combinations(range(n), o)]
        self.ns = len(self.strings)
        self.sidx = {s: k for k, s in enumerate(self.strings)}
        self.dim = self.ns * self.ns
        hf_string = (1 << o) - 1
        self.hf = self.sidx[hf_string] * self.ns + self.sidx[hf_string]
        # single-string excitation tables: exc[p][q] = list of (src, dst, sign)
        self.exc = [[[] for _ in range(n)] for _ in range(n)]
        for k, s in enumerate(self.strings):
            for q in range(n):
                if not (s >> q) & 1:
                    continue
                s1 = s ^ (1 << q)
                sg1 = -1 if _popcount(s & ((1 << q) - 1)) % 2 else 1
                for p in range(n):
                    if (s1 >> p) & 1:
                        continue
                    s2 = s1 | (1 << p)
                    sg2 = -1 if _popcount(s1 & ((1 << p) - 1)) % 2 else 1
                    self.exc[p][q].append((k, self.sidx[s2], sg1 * sg2))
        self._E = {}

    # -- operators ---------------------------------------------------------
    def E(self, p: int, q: int) -> np.ndarray:
        """Dense matrix of the singlet excitation operator E_pq."""
        key = (p, q)
        if key not in self._E:
            m = np.zeros((self.dim, self.dim))
            ns = self.ns
            for (src, dst, sg) in self.exc[p][q]:
                # alpha part: (src, b) -> (dst, b)
                for b in range(ns):
                    m[dst * ns + b, src * ns + b] += sg
                # beta part: (a, src) -> (a, dst)
                for a in range(ns):
                    m[a * ns + dst, a * ns + src] += sg
            self._E[key] = m
        return self._E[key]

    def hamiltonian(self, h: np.ndarray, g: np.ndarray) -> np.ndarray:
        """H = sum h_pq E_pq + 1/2 sum g_pqrs (E_pq E_rs - delta_qr E_ps); g in Mulliken order."""
        n = self.n
        H = np.zeros((self.dim, self.dim))
        for p in range(n):
            for q in range(n):
                Epq = self.E(p, q)
                coef = h[p, q] - 0.5 * sum(g[p, r, r, q] for r in range(n))
                H += coef * Epq
                K = np.zeros_like(H)
                for r in range(n):
                    for s in range(n):
                        if g[p, q, r, s] != 0.0:
                            K += g[p, q, r, s] * self.E(r, s)
                H += 0.5 * Epq @ K
        return H

    # -- excitation manifold -------------------------------------------------
    def singles_index(self):
        o, v = self.o, self.v
        return [(i, a) for i in range(o) for a in range(v)]

    def doubles_packed(self):
        """Packed doubles (p, q) with p >= q over compound singles indices."""
        s = self.singles_index()
        return [(p, q) for p in range(len(s)) for q in range(p + 1)]

    def tau_single(self, i: int, a: int) -> np.ndarray:
        return self.E(self.o + a, i)

    def operator(self, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
        """X = sum x1[i,a] E_ai + 1/2 sum x2[i,j,a,b] E_ai E_bj as a dense matrix."""
        o, v = self.o, self.v
        X = np.zeros((self.dim, self.dim))
        for i in range(o):
            for a in range(v):
                if x1[i, a] != 0.0:
                    X += x1[i, a] * self.tau_single(i, a)
        for i in range(o):
            for a in range(v):
                Eai = self.tau_single(i, a)
                for j in range(o):
                    for b in range(v):
                        c = x2[i, j, a, b]
                        if c != 0.0:
                            X += 0.5 * c * (Eai @ self.tau_single(j, b))
        return X

    def manifold(self):
        """Columns tau_mu|HF> of the packed manifold and the biorthonormal bra rows."""
        if hasattr(self, "_V"):
            return self._V, self._Vp
        hf = np.zeros(self.dim)
        hf[self.hf] = 1.0
        cols = []
        s = self.singles_index()
        for (i, a) in s:
            cols.append(self.tau_single(i, a) @ hf)
        for (p, q) in self.doubles_packed():
            (i, a), (j, b) = s[p], s[q]
            vec = self.tau_single(i, a) @ (self.tau_single(j, b) @ hf)
            if p == q:
                vec = 0.5 * vec
            cols.append(vec)
        V = np.array(cols).T
        Vp = np.linalg.solve(V.T @ V, V.T)
        self._V, self._Vp = V, Vp
        return V, Vp

    def hf_vector(self) -> np.ndarray:
        e = np.zeros(self.dim)
        e[self.hf] = 1.0
        return e

    def unpack(self, packed: np.ndarray):
        """Packed manifold coefficients -> (x1[i,a], x2[i,j,a,b])."""
        o, v = self.o, self.v
        s = self.singles_index()
        ns1 = len(s)
        x1 = np.zeros((o, v))
        x2 = np.zeros((o, o, v, v))
        for k, (i, a) in enumerate(s):
            x1[i, a] = packed[k]
        for k, (p, q) in enumerate(self.doubles_packed()):
            (i, a), (j, b) = s[p], s[q]
            x2[i, j, a, b] = packed[ns1 + k]
            x2[j, i, b, a] = packed[ns1 + k]
        return x1, x2

    def pack(self, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
        s = self.singles_index()
        out = [x1[i, a] for (i, a) in s]
        for (p, q) in self.doubles_packed():
            (i, a), (j, b) = s[p], s[q]
            out.append(x2[i, j, a, b])
        return np.array(out)


def expm_nilpotent(T: np.ndarray, order: int) -> np.ndarray:
    """exp(T) by its Taylor series; exact when T^(order+1) = 0."""
    out = np.eye(T.shape[0])
    term = np.eye(T.shape[0])
    for k in range(1, order + 1):
        term = term @ T / k
        out = out + term
    return out


class CCBruteForce:
    """All CC quantities of the Theory section evaluated literally in Fock space."""

    def __init__(self, h: np.ndarray, B: np.ndarray, o: int):
        self.n = h.shape[0]
        self.o, self.v = o, self.n - o
        self.fs = FockSpace(self.n, o)
        g = np.einsum("Ppq,Prs->pqrs", B, B)
        self.H = self.fs.hamiltonian(h, g)
        self.order = 2 * o + 1

    def hbar(self, t1, t2, H=None):
        H = self.H if H is None else H
        T = self.fs.operator(t1, t2)
        return expm_nilpotent(-T, self.order) @ H @ expm_nilpotent(T, self.order)

    def residual(self, t1, t2):
        """(Omega1, Omega2, E) = (<mu~|Hbar|HF> unpacked, <HF|Hbar|HF>)."""
        V, Vp = self.fs.manifold()
        Hb = self.hbar(t1, t2)
        hf = self.fs.hf_vector()
        vec = Hb @ hf
        om = Vp @ vec
        o1, o2 = self.fs.unpack(om)
        return o1, o2, float(hf @ vec)

    def hamiltonian_derivative(self, h1, B, B1):
        g1 = np.einsum("Ppq,Prs->pqrs", B1, B) + np.einsum("Ppq,Prs->pqrs", B, B1)
        return self.fs.hamiltonian(h1, g1)

    def residual_x(self, t1, t2, Hx):
        """<mu~|exp(-T) H^x exp(T)|HF> for a Hamiltonian derivative H^x."""
        V, Vp = self.fs.manifold()
        Hb = self.hbar(t1, t2, Hx)
        hf = self.fs.hf_vector()
        vec = Hb @ hf
        o1, o2 = self.fs.unpack(Vp @ vec)
        return o1, o2, float(hf @ vec)

    def jacobian_right(self, t1, t2, r1, r2):
        """A R = <mu~|[Hbar, R]|HF>."""
        V, Vp = self.fs.manifold()
        Hb = self.hbar(t1, t2)
        R = self.fs.operator(r1, r2)
        hf = self.fs.hf_vector()
        return self.fs.unpack(Vp @ ((Hb @ R - R @ Hb) @ hf))

    def left_bra(self, l0, l1, l2):
        """<L| = l0 <HF| + sum_mu L_mu <mu~| as a row vector."""
        V, Vp = self.fs.manifold()
        return l0 * self.fs.hf_vector() + self.fs.pack(l1, l2) @ Vp

    def jacobian_left(self, t1, t2, l1, l2):
        """(L^T A)_nu = <L|[Hbar, tau_nu]|HF> for every packed nu, returned unpacked."""
        Hb = self.hbar(t1, t2)
        bra = self.left_bra(0.0, l1, l2)
        hf = self.fs.hf_vector()
        V, _ = self.fs.manifold()
        out = []
        s = self.fs.singles_index()
        for k in range(V.shape[1]):
            tau = self._tau(k)
            out.append(bra @ ((Hb @ tau - tau @ Hb) @ hf))
        return self.fs.unpack(np.array(out))

    def _tau(self, k: int) -> np.ndarray:
        s = self.fs.singles_index()
        if k < len(s):
            i, a = s[k]
            return self.fs.tau_single(i, a)
        p, q = self.fs.doubles_packed()[k - len(s)]
        (i, a), (j, b) = s[p], s[q]
        m = self.fs.tau_single(i, a) @ self.fs.tau_single(j, b)
        return 0.5 * m if p == q else m

    def eta(self, t1, t2):
        """eta_nu = <HF|[Hbar, tau_nu]|HF>."""
        Hb = self.hbar(t1, t2)
        hf = self.fs.hf_vector()
        V, _ = self.fs.manifold()
        out = [hf @ ((Hb @ self._tau(k) - self._tau(k) @ Hb) @ hf) for k in range(V.shape[1])]
        return self.fs.unpack(np.array(out))

    def fmatrix(self, t1, t2, g0, g1, g2, r1, r2):
        """(F(g) R)_mu = <g|[[Hbar, tau_mu], R]|HF> with <g| = g0<HF| + sum g_nu <nu~|."""
        Hb = self.hbar(t1, t2)
        bra = self.left_bra(g0, g1, g2)
        R = self.fs.operator(r1, r2)
        hf = self.fs.hf_vector()
        V, _ = self.fs.manifold()
        out = []
        for k in range(V.shape[1]):
            tau = self._tau(k)
            c1 = Hb @ tau - tau @ Hb
            c2 = c1 @ R - R @ c1
            out.append(bra @ (c2 @ hf))
        return self.fs.unpack(np.array(out))

    def state_right(self, t1, t2, r0, r1, r2):
        """|psi^R> = (r0 + R) exp(T)|HF> as a determinant-space vector."""
        T = self.fs.operator(t1, t2)
        R = self.fs.operator(r1, r2)
        v = expm_nilpotent(T, self.order) @ self.fs.hf_vector()
        return r0 * v + R @ v

    def state_left(self, t1, t2, l0, l1, l2):
        """<psi^L| = <HF|(l0 + L) exp(-T) as a determinant-space row vector."""
        T = self.fs.operator(t1, t2)
        return self.left_bra(l0, l1, l2) @ expm_nilpotent(-T, self.order)

    def tau_expectation(self, l0, l1, l2, r0, r1, r2):
        """<L|tau_sigma|R> = <L|tau_sigma (r0 + R)|HF> for every packed sigma, unpacked."""
        bra = self.left_bra(l0, l1, l2)
        R = self.fs.operator(r1, r2)
        ket = r0 * self.fs.hf_vector() + R @ self.fs.hf_vector()
        V, _ = self.fs.manifold()
        out = [bra @ (self._tau(k) @ ket) for k in range(V.shape[1])]
        return self.fs.unpack(np.array(out))

    def overlap_shifted(self, l0, l1, l2, r0, r1, r2, d1, d2):
        """<L|(r0 + R) exp(D)|HF> for amplitude shifts D = (d1, d2)."""
        bra = self.left_bra(l0, l1, l2)
        R = self.fs.operator(r1, r2)
        Dm = self.fs.operator(d1, d2)
        ket = expm_nilpotent(Dm, self.order) @ self.fs.hf_vector()
        return float(bra @ (r0 * ket + R @ ket))

    def fci(self):
        """Eigenpairs of H restricted to singlets (S^2 = 0), ascending energies."""
        w, U = np.linalg.eigh(self.H)
        S2 = self._s2()
        keep = [k for k in range(len(w)) if abs(U[:, k] @ S2 @ U[:, k]) < 1e-8]
        return w[keep], U[:, keep]

    def _s2(self):
        """S^2 in the determinant space, built from spin-orbital ladder operators."""
        if hasattr(self, "_S2"):
            return self._S2
        fs = self.fs
        n, ns = fs.n, fs.ns
        # S+ = sum_p a+_pa a_pb ; S- = S+^T ; Sz = (Na - Nb)/2 = 0 in this space
        # S^2 = S- S+ + Sz(Sz+1) = S- S+ here.  Build S+ as a map into the
        # (o+1, o-1) space, represented through explicit string tables.
        o = fs.o
        up_strings = [sum(1 << p for p in c) for c in itertools.combinations(range(n), o + 1)] if o + 1 <= n else []
        dn_strings = [sum(1 << p for p in c) for c in itertools.combinations(range(n), o - 1)] if o >= 1 else []
        uidx = {s: k for k, s in enumerate(up_strings)}
        didx = {s: k for k, s in enumerate(dn_strings)}
        Sp = np.zeros((len(up_strings) * len(dn_strings), fs.dim))
        for ka, sa in enumerate(fs.strings):
            for kb, sb in enumerate(fs.strings):
                col = ka * ns + kb
                for p in range(n):
                    if not (sb >> p) & 1 or (sa >> p) & 1:
                        continue
                    # a_pb acts first (beta bits sit above all alpha bits: o alpha bits
                    # precede, plus beta bits below p), then a+_pa (alpha bits below p)
                    sgn_b = (-1) ** (o + _popcount(sb & ((1 << p) - 1)))
                    sb2 = sb ^ (1 << p)
                    sgn_a = (-1) ** _popcount(sa & ((1 << p) - 1))
                    sa2 = sa | (1 << p)
                    # after removing the beta electron the alpha string gains one
                    # electron; the beta block offset changes by one electron, which
                    # is a common phase for all terms and does not affect S^2.
                    row = uidx[sa2] * len(dn_strings) + didx[sb2]
                    Sp[row, col] += sgn_a * sgn_b
        self._S2 = Sp.T @ Sp
        return self._S2


def hamiltonian_matrix_elements_check(n: int, o: int) -> int:
    """Number of determinants, for sizing tests."""
    return math.comb(n, o) ** 2
