"""Ground state, multipliers, EOM states and derivative couplings (oracle).

Test infrastructure of the oracle; see the package docstring.  Everything is
FP64 on the CPU and built on :mod:`oracle.ccsd`.

Paper passages followed:
* amplitude equations Omega(t) = 0 and E = <HF|Hbar|HF> (Theory, Lagrangian);
* ground-state left state <psi_0^L| = <HF|(1 + Lambda) exp(-T) with
  lambda^T A = -eta^T (the j = 0 analogue of the multiplier equations);
* EOM states A R_k = omega_k R_k, L_k^T A = omega_k L_k^T, L_k^T R_l = delta_kl,
  L_0^k = 0 and R_0^k = eta^T R_k / omega_k (the state parametrisation with
  R_0^k and L_0^k; the value of R_0^k follows from the reference row of the
  EOM eigenproblem, which the paper does not print);
* coupling multipliers gamma = L_i / (omega_j - omega_i) (Eq. for gamma),
  t-eta (Eq. for t-eta and its CCSD first term), zeta^T A = -t-eta^T (Eq.
  amplituderelax), and F^q = <L_i|[Hbar^q, R_j]|HF>/(omega_j - omega_i) +
  <zeta|Hbar^q|HF> (Eq. NAC_NC) with the orbital term absent because the
  orbitals are fixed and x-independent (the relaxed-orbital form, with HF
  orbitals that follow x, is in relaxed.py); for j = 0, zeta = L_i/(E_0 - E_i) and
  F_i0 = <zeta|Hbar^q|HF> (Eqs. for the ground-state right state);
* the definition F_ij = <psi_i^L | d/dx psi_j^R> (Eq. nac), evaluated by central
  differences of O_ij(x) = <psi_i^L(x0)|psi_j^R(x)> with the normalisation
  L_j(x0)^T R_j(x) = 1 fixed by the xi condition of the Lagrangian.

Reading used for i = 0 (paper silent): the left ground state is
<HF|(1 + Lambda), so in gamma, in t-eta's F-matrix term and in the first term
of Eq. NAC_NC the reference component 1 enters as well, multiplying the
energy derivatives (<HF|[[Hbar,tau],tau]|HF> and <HF|[Hbar^q, R_j]|HF>), with
omega_0 = 0.  The finite-difference test checks this reading.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import ccsd as cc

F64 = torch.float64


# ---------------------------------------------------------------------------
# vectors
# ---------------------------------------------------------------------------

def packed_indices(o: int, v: int):
    """Storage positions of the packed manifold: singles (i,a), doubles (ia) >= (jb)."""
    s = [(i, a) for i in range(o) for a in range(v)]
    d = [(p, q) for p in range(len(s)) for q in range(p + 1)]
    return s, d


def pack(x1, x2):
    o, v = x1.shape
    s, d = packed_indices(o, v)
    ii = torch.tensor([s[p][0] for p, q in d], dtype=torch.long)
    aa = torch.tensor([s[p][1] for p, q in d], dtype=torch.long)
    jj = torch.tensor([s[q][0] for p, q in d], dtype=torch.long)
    bb = torch.tensor([s[q][1] for p, q in d], dtype=torch.long)
    return torch.cat([x1.reshape(-1), x2[ii, jj, aa, bb]])


def unpack(x, o, v):
    s, d = packed_indices(o, v)
    ns = o * v
    x1 = x[:ns].reshape(o, v).clone()
    x2 = torch.zeros((o, o, v, v), dtype=F64)
    ii = torch.tensor([s[p][0] for p, q in d], dtype=torch.long)
    aa = torch.tensor([s[p][1] for p, q in d], dtype=torch.long)
    jj = torch.tensor([s[q][0] for p, q in d], dtype=torch.long)
    bb = torch.tensor([s[q][1] for p, q in d], dtype=torch.long)
    x2[ii, jj, aa, bb] = x[ns:]
    x2[jj, ii, bb, aa] = x[ns:]
    return x1, x2


def packed_dim(o, v):
    return o * v + o * v * (o * v + 1) // 2


def denominators(eps, o):
    e = cc.as_t(eps)
    eo, ev = e[:o], e[o:]
    d1 = ev[None, :] - eo[:, None]
    d2 = d1[:, None, :, None] + d1[None, :, None, :]
    return d1, d2


class Vec:
    """A (singles, doubles) pair with the packed inner product."""

    __slots__ = ("x1", "x2")

    def __init__(self, x1, x2):
        self.x1, self.x2 = x1, x2

    def __add__(self, o):
        return Vec(self.x1 + o.x1, self.x2 + o.x2)

    def __sub__(self, o):
        return Vec(self.x1 - o.x1, self.x2 - o.x2)

    def __mul__(self, s):
        return Vec(self.x1 * s, self.x2 * s)

    __rmul__ = __mul__

    def __truediv__(self, s):
        return Vec(self.x1 / s, self.x2 / s)

    def div(self, d1, d2):
        return Vec(self.x1 / d1, self.x2 / d2)

    def dot(self, o):
        return float(cc.pdot(self.x1, self.x2, o.x1, o.x2))

    def norm(self):
        return self.dot(self) ** 0.5

    def maxabs(self):
        return max(float(self.x1.abs().max()), float(self.x2.abs().max()))

    def copy(self):
        return Vec(self.x1.clone(), self.x2.clone())

    @staticmethod
    def zeros(o, v):
        return Vec(torch.zeros((o, v), dtype=F64), torch.zeros((o, o, v, v), dtype=F64))


class DIIS:
    """Pulay extrapolation over (vector, error) pairs with the packed inner product."""

    def __init__(self, dim: int = 8):
        self.dim = dim
        self.vecs, self.errs = [], []

    def __call__(self, x: Vec, e: Vec) -> Vec:
        self.vecs.append(x)
        self.errs.append(e)
        if len(self.vecs) > self.dim:
            self.vecs.pop(0)
            self.errs.pop(0)
        m = len(self.vecs)
        if m < 2:
            return x
        Bm = np.zeros((m + 1, m + 1))
        for a in range(m):
            for b in range(a + 1):
                Bm[a, b] = Bm[b, a] = self.errs[a].dot(self.errs[b])
        Bm[m, :m] = Bm[:m, m] = -1.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        scale = np.abs(np.diag(Bm[:m, :m])).max()
        Bs = Bm.copy()
        Bs[:m, :m] /= scale
        try:
            c = np.linalg.solve(Bs, rhs)[:m]
        except np.linalg.LinAlgError:
            return x
        out = self.vecs[0] * c[0]
        for a in range(1, m):
            out = out + self.vecs[a] * c[a]
        return out


# ---------------------------------------------------------------------------
# the system
# ---------------------------------------------------------------------------

@dataclass
class State:
    """A CC state: (r0, R) for right states, (l0, L) for left states."""
    c0: float
    vec: Vec


@dataclass
class Result:
    e_ccsd: float = 0.0
    t: Vec | None = None
    lam: Vec | None = None
    omega: list = field(default_factory=list)
    right: list = field(default_factory=list)   # State per excited root (r0, R)
    left: list = field(default_factory=list)    # State per excited root (0, L)
    iters: dict = field(default_factory=dict)


class System:
    """The oracle's view of one closed-shell Hamiltonian (h, B) with o occupied orbitals."""

    def __init__(self, eps, h, B, o, vvvv_batch=None):
        self.eps = cc.as_t(eps)
        self.h = cc.as_t(h)
        self.B = cc.as_t(B)
        self.o = o
        self.n = self.h.shape[0]
        self.v = self.n - o
        self.kw = {} if vvvv_batch is None else {"vvvv_batch": vvvv_batch}
        self.d1, self.d2 = denominators(self.eps, o)

    # basic maps --------------------------------------------------------
    def residual(self, t: Vec):
        o1, o2, e = cc.residual(t.x1, t.x2, self.h, self.B, self.o, **self.kw)
        return Vec(o1, o2), float(e)

    def right(self, t: Vec, r: Vec) -> Vec:
        return Vec(*cc.jacobian_right(t.x1, t.x2, r.x1, r.x2, self.h, self.B, self.o, **self.kw))

    def left(self, t: Vec, l: Vec) -> Vec:
        return Vec(*cc.jacobian_left(t.x1, t.x2, l.x1, l.x2, self.h, self.B, self.o, **self.kw))

    def eta(self, t: Vec) -> Vec:
        return Vec(*cc.eta(t.x1, t.x2, self.h, self.B, self.o, **self.kw))

    def hess_right(self, t: Vec, g0: float, g: Vec, r: Vec) -> Vec:
        return Vec(*cc.lagrangian_hessian_right(t.x1, t.x2, g0, g.x1, g.x2, r.x1, r.x2,
                                                self.h, self.B, self.o, **self.kw))

    def precond(self, x: Vec, shift: float = 0.0) -> Vec:
        return Vec(x.x1 / (self.d1 - shift), x.x2 / (self.d2 - shift))

    # ground state ---------------------------------------------------------
    def solve_ground(self, tol=1e-11, maxit=200, diis_dim=8, t0: Vec | None = None):
        t = Vec.zeros(self.o, self.v) if t0 is None else t0.copy()
        diis = DIIS(diis_dim)
        for it in range(1, maxit + 1):
            om, e = self.residual(t)
            if om.maxabs() < tol:
                return t, e, it
            t = diis(t - self.precond(om), om)
        raise RuntimeError("ground state not converged")

    def solve_left_linear(self, t: Vec, rhs: Vec, tol=1e-10, maxit=200, diis_dim=8, x0=None):
        """Solve x^T A = -rhs^T (Eq. amplituderelax form) by preconditioned DIIS."""
        x = self.precond(rhs) * (-1.0) if x0 is None else x0.copy()
        diis = DIIS(diis_dim)
        for it in range(1, maxit + 1):
            res = rhs + self.left(t, x)
            if res.maxabs() < tol:
                return x, it
            x = diis(x - self.precond(res), res)
        raise RuntimeError("left linear equations not converged")

    def solve_lambda(self, t: Vec, tol=1e-10, **kw):
        return self.solve_left_linear(t, self.eta(t), tol=tol, **kw)

    # EOM ----------------------------------------------------------------
    def dense_jacobian(self, t: Vec) -> torch.Tensor:
        """A in packed coordinates, column by column (small systems only)."""
        n = packed_dim(self.o, self.v)
        A = torch.zeros((n, n), dtype=F64)
        for k in range(n):
            e = torch.zeros(n, dtype=F64)
            e[k] = 1.0
            r = Vec(*unpack(e, self.o, self.v))
            ar = self.right(t, r)
            A[:, k] = pack(ar.x1, ar.x2)
        return A

    def eom_dense(self, t: Vec, nroots: int):
        A = self.dense_jacobian(t).numpy()
        w, Vr = np.linalg.eig(A)
        order = np.argsort(w.real)[:nroots]
        if np.abs(w[order].imag).max() > 1e-10:
            raise RuntimeError("complex root among the wanted roots")
        wl, Vl = np.linalg.eig(A.T)
        orderl = np.argsort(wl.real)[:nroots]
        omega = w[order].real
        R = [Vec(*unpack(torch.as_tensor(Vr[:, k].real), self.o, self.v)) for k in order]
        L = [Vec(*unpack(torch.as_tensor(Vl[:, k].real), self.o, self.v)) for k in orderl]
        return omega, R, L

    def davidson(self, apply, nroots, tol=1e-9, maxit=200, maxsub=None, guesses=None, max_complex=12):
        """Block Davidson for the lowest nroots (by real part) of a non-symmetric map.

        A small subspace of a non-symmetric map can give a complex-conjugate pair of
        Ritz values among the wanted ones even when the converged roots are real.
        Such a pair is treated as transient: the subspace is expanded with the
        preconditioned real and imaginary parts of the pair's residual (the real
        2-D invariant subspace of the pair), and the solve fails only when a
        complex pair stays among the wanted roots for more than `max_complex`
        consecutive expansions.  A complex wanted root never counts as converged.
        When the subspace would exceed maxsub it restarts from the current and the
        previous Ritz vectors (their images carried along, no transforms).
        """
        o, v = self.o, self.v
        maxsub = maxsub or max(8 * nroots, 24)
        if guesses is None:
            order = torch.argsort(self.d1.reshape(-1))[:nroots]
            guesses = []
            for k in order:
                g = Vec.zeros(o, v)
                g.x1.view(-1)[k] = 1.0
                guesses.append(g)
        V, AV = [], []

        def add(x):
            x = x / x.norm()
            for _ in range(2):
                for b in V:
                    x = x - b * b.dot(x)
            nrm = x.norm()
            if nrm < 1e-8:
                return False
            x = x / nrm
            V.append(x)
            AV.append(apply(x))
            return True

        def add_known(x, ax):
            # as add, for a vector whose image ax = A x is known: the same combination applied to
            # ax gives the image of the orthonormalised vector, without another transform
            n0 = x.norm()
            x, ax = x / n0, ax / n0
            for _ in range(2):
                for b, ab in zip(V, AV):
                    c = b.dot(x)
                    x, ax = x - b * c, ax - ab * c
            nrm = x.norm()
            if nrm < 1e-8:
                return False
            V.append(x / nrm)
            AV.append(ax / nrm)
            return True

        def combine(basis, u):
            x = basis[0] * u[0]
            for a in range(1, len(basis)):
                x = x + basis[a] * u[a]
            return x

        for g in guesses:
            add(g)
        n_complex = 0
        prev = []  # the previous iteration's Ritz vectors and their images
        for it in range(1, maxit + 1):
            m = len(V)
            G = np.array([[V[a].dot(AV[b]) for b in range(m)] for a in range(m)])
            w, U = np.linalg.eig(G)
            order = np.argsort(w.real)[:nroots]
            is_complex = np.abs(w[order].imag) > 1e-8
            n_complex = n_complex + 1 if is_complex.any() else 0
            if n_complex > max_complex:
                raise RuntimeError("complex root among the wanted roots")
            X, AX, res, ok = [], [], [], not is_complex.any()
            for k in order:
                wr, wi = w[k].real, w[k].imag
                ur, ui = U[:, k].real, U[:, k].imag
                xr, axr = combine(V, ur), combine(AV, ur)
                if abs(wi) <= 1e-8:
                    r = axr - xr * wr
                    X.append(xr)
                    AX.append(axr)
                    res.append((r, wr))
                    if r.norm() > tol:
                        ok = False
                    continue
                # complex Ritz pair: A(xr + i xi) - (wr + i wi)(xr + i xi), real and imaginary parts
                xi, axi = combine(V, ui), combine(AV, ui)
                X.extend([xr, xi])
                AX.extend([axr, axi])
                res.append((axr - xr * wr + xi * wi, wr))
                res.append((axi - xi * wr - xr * wi, wr))
            if ok:
                return np.array([w[k].real for k in order]), X, it
            if m + len(res) > maxsub:
                # thick restart: the Ritz vectors and those of the previous iteration (the last
                # search directions, which a restart to the Ritz vectors alone discards and which
                # carry the convergence of a non-symmetric matrix), with their known images
                V.clear()
                AV.clear()
                for x, ax in list(zip(X, AX)) + prev:
                    add_known(x, ax)
            prev = list(zip(X, AX))
            for (r, wk) in res:
                if r.norm() > tol:
                    add(self.precond(r, wk))
        raise RuntimeError("Davidson not converged")

    @staticmethod
    def normalize_right(R: Vec) -> Vec:
        """||R|| = 1 (packed norm); the component of largest magnitude is positive.

        The search runs over singles then doubles in storage order and the first
        maximum wins.
        """
        R = R / R.norm()
        flat = torch.cat([R.x1.reshape(-1), R.x2.reshape(-1)])
        k = int(torch.argmax(flat.abs()))
        if float(flat[k]) < 0:
            R = R * -1.0
        return R

    def eom(self, t: Vec, nroots: int, dense=False, tol=1e-9):
        if dense:
            omega, R, L = self.eom_dense(t, nroots)
            return self.eom_from_vectors(t, omega, R, omega, L)
        omega, R, _ = self.davidson(lambda x: self.right(t, x), nroots, tol=tol)
        omega_l, L, _ = self.davidson(lambda x: self.left(t, x), nroots, tol=tol)
        return self.eom_from_vectors(t, omega, R, omega_l, L)

    def eom_from_vectors(self, t: Vec, omega, R, omega_l, L):
        """Biorthonormal states from right and left eigenvectors of the same roots."""
        nroots = len(R)
        if np.abs(np.asarray(omega) - np.asarray(omega_l)).max() > 1e-6:
            raise RuntimeError("left and right EOM roots differ")
        R = [self.normalize_right(r) for r in R]
        # biorthonormalise: L_k^T R_l = delta_kl (roots are non-degenerate).
        # With M[m, l] = <L_m|R_l> and L'_k = sum_m c[m, k] L_m, <L'_k|R_l> = (c^T M)[k, l],
        # so c = M^{-T}.
        M = np.array([[L[k].dot(R[l]) for l in range(nroots)] for k in range(nroots)])
        c = np.linalg.inv(M).T
        Lnew = []
        for k in range(nroots):
            x = L[0] * c[0, k]
            for m in range(1, nroots):
                x = x + L[m] * c[m, k]
            Lnew.append(x)
        eta = self.eta(t)
        right = [State(eta.dot(R[k]) / omega[k], R[k]) for k in range(nroots)]
        left = [State(0.0, Lnew[k]) for k in range(nroots)]
        return list(omega), right, left

    # full pipeline --------------------------------------------------------
    def run(self, nroots: int, dense=False, tol=1e-11, tol_eom=1e-9, tol_lin=1e-10):
        res = Result()
        t, e, it = self.solve_ground(tol=tol)
        res.t, res.e_ccsd, res.iters["ground"] = t, e, it
        res.lam, res.iters["lambda"] = self.solve_lambda(t, tol=tol_lin)
        if nroots > 0:
            res.omega, res.right, res.left = self.eom(t, nroots, dense=dense, tol=tol_eom)
        return res

    def left_state(self, res: Result, i: int) -> State:
        return State(1.0, res.lam) if i == 0 else res.left[i - 1]

    def right_state(self, res: Result, j: int) -> State:
        if j == 0:
            return State(1.0, Vec.zeros(self.o, self.v))
        return res.right[j - 1]

    def omega_of(self, res: Result, k: int) -> float:
        return 0.0 if k == 0 else res.omega[k - 1]

    # couplings ---------------------------------------------------------
    def overlap(self, L: State, R: State, d: Vec) -> torch.Tensor:
        """<L|(r0 + R) exp(D)|HF> projected on <= doubles (L de-excites at most twice)."""
        r0, r1, r2 = R.c0, R.vec.x1, R.vec.x2
        d1, d2 = d.x1, d.x2
        c1 = r0 * d1 + r1
        dd = torch.einsum("ia,jb->ijab", d1, d1)
        rd = torch.einsum("ia,jb->ijab", r1, d1)
        c2 = r0 * (d2 + dd) + rd + rd.permute(1, 0, 3, 2) + r2
        return L.c0 * r0 + cc.pdot(L.vec.x1, L.vec.x2, c1, c2)

    def tau_expectation(self, L: State, R: State) -> Vec:
        """<L|tau_sigma|R> for every packed sigma: the gradient of the overlap at D = 0."""
        z1 = torch.zeros((self.o, self.v), dtype=F64)
        z2 = torch.zeros((self.o, self.o, self.v, self.v), dtype=F64)
        g1, g2 = torch.func.grad(lambda a, b: self.overlap(L, R, Vec(a, b)), argnums=(0, 1))(z1, z2)
        return Vec(*cc.packed_grad(g1, g2))

    def coupling_multipliers(self, res: Result, i: int, j: int, tol_lin=1e-10):
        """(g0, gamma, zeta) for the pair (i, j), i != j."""
        t = res.t
        Li = self.left_state(res, i)
        if j == 0:
            if i == 0:
                raise ValueError("i == j")
            zeta = Li.vec * (-1.0 / res.omega[i - 1])
            return 0.0, Vec.zeros(self.o, self.v), zeta
        Rj = self.right_state(res, j)
        dw = self.omega_of(res, j) - self.omega_of(res, i)
        g0 = Li.c0 / dw
        gam = Li.vec / dw
        teta = self.tau_expectation(Li, Rj) + self.hess_right(t, g0, gam, Rj.vec)
        zeta, _ = self.solve_left_linear(t, teta, tol=tol_lin)
        return g0, gam, zeta

    def coupling(self, res: Result, i: int, j: int, h1, B1, tol_lin=1e-10):
        """F_ij^x of Eq. NAC_NC (orbital term absent: orbitals fixed) along (h1, B1)."""
        h1, B1 = cc.as_t(h1), cc.as_t(B1)
        t = res.t
        g0, gam, zeta = self.coupling_multipliers(res, i, j, tol_lin)
        ox1, ox2, _ = cc.hamiltonian_derivative_residual(t.x1, t.x2, self.h, self.B, h1, B1, self.o, **self.kw)
        f = zeta.dot(Vec(ox1, ox2))
        if j > 0:
            Rj = self.right_state(res, j)
            x1, x2, xe = cc.hamiltonian_derivative_jacobian(t.x1, t.x2, Rj.vec.x1, Rj.vec.x2,
                                                            self.h, self.B, h1, B1, self.o, **self.kw)
            f += g0 * float(xe) + gam.dot(Vec(x1, x2))
        return f

    # state energy gradients ------------------------------------------------
    def energy_gradient(self, res: Result, k: int, h1, B1, tol_lin=1e-10):
        """dE_k/dx along (h1, B1), orbitals fixed, from the energy Lagrangian.

        The same construction as the coupling Lagrangian (Lagrangian section) with the
        state energy in place of the overlap: E_0 + lambda.Omega for the ground state
        (lambda^T A = -eta); for k >= 1, E_k = E_0 + omega_k and omega_k = L_k.(A R_k) is
        stationary in L_k and R_k (biorthonormal eigenvectors, L_k.R_k = 1), so only its
        amplitude dependence needs a multiplier: zeta^T A = -(F(L_k) R_k), and
        domega_k/dx = L_k.(A^x R_k) + zeta.Omega^x at fixed t, L_k, R_k.
        """
        return self.energy_lagrangian_derivative(res, k, self.energy_multiplier(res, k, tol_lin), h1, B1)

    def energy_multiplier(self, res: Result, k: int, tol_lin=1e-10):
        """zeta of the excited-state energy Lagrangian, zeta^T A = -(F(L_k) R_k); None for k = 0."""
        if k == 0:
            return None
        L, R = res.left[k - 1].vec, res.right[k - 1].vec
        zeta, _ = self.solve_left_linear(res.t, self.hess_right(res.t, 0.0, L, R), tol=tol_lin)
        return zeta

    def energy_lagrangian_derivative(self, res: Result, k: int, zeta, dh, dB) -> float:
        """Derivative of the energy Lagrangian of state k along (dh, dB) at fixed amplitudes and
        multipliers: E^x + lambda.Omega^x, plus L_k.(A^x R_k) + zeta.Omega^x for k >= 1."""
        dh, dB = cc.as_t(dh), cc.as_t(dB)
        t = res.t
        ox1, ox2, oe = cc.hamiltonian_derivative_residual(t.x1, t.x2, self.h, self.B, dh, dB, self.o, **self.kw)
        om_x = Vec(ox1, ox2)
        g = float(oe) + float(res.lam.dot(om_x))
        if k > 0:
            L, R = res.left[k - 1].vec, res.right[k - 1].vec
            x1, x2, _ = cc.hamiltonian_derivative_jacobian(t.x1, t.x2, R.x1, R.x2, self.h, self.B, dh, dB,
                                                           self.o, **self.kw)
            g += float(L.dot(Vec(x1, x2))) + float(zeta.dot(om_x))
        return g

    def energy_at(self, res0: Result, k: int, x: float, h1, B1, tol=1e-12):
        """E_k(x): ground state from t(x0), root k matched by the largest |L_k(x0).R(x)|."""
        sx = self.displaced(x, h1, B1)
        tx, ex, _ = sx.solve_ground(tol=tol, t0=res0.t)
        if k == 0:
            return float(ex)
        omega, R, _ = sx.eom_dense(tx, len(res0.omega) + 2)
        Lk = res0.left[k - 1].vec
        j = int(np.argmax([abs(Lk.dot(r)) for r in R]))
        return float(ex) + float(omega[j])

    def energy_gradient_fd(self, res0: Result, k: int, h1, B1, delta=2e-3):
        """Central differences of E_k(x) with one Richardson step: error O(delta^4)."""
        E = {s: self.energy_at(res0, k, s * delta, h1, B1) for s in (-2, -1, 1, 2)}
        return (8.0 * (E[1] - E[-1]) - (E[2] - E[-2])) / (12.0 * delta)

    # finite differences of the definition ----------------------------------
    def displaced(self, x, h1, B1):
        return System(self.eps, self.h + x * cc.as_t(h1), self.B + x * cc.as_t(B1), self.o,
                      vvvv_batch=self.kw.get("vvvv_batch"))

    def overlap_at(self, res0: Result, i: int, j: int, x: float, h1, B1, tol=1e-12):
        """O_ij(x) = <psi_i^L(x0)|psi_j^R(x)> with L_j(x0)^T R_j(x) = 1."""
        sx = self.displaced(x, h1, B1)
        tx, _, _ = sx.solve_ground(tol=tol, t0=res0.t)
        Li = self.left_state(res0, i)
        if j == 0:
            Rx = State(1.0, Vec.zeros(self.o, self.v))
        else:
            nroots = len(res0.omega)
            omega, R, _ = sx.eom_dense(tx, nroots + 2)
            Lj = res0.left[j - 1].vec
            ov = [abs(Lj.dot(r)) for r in R]
            k = int(np.argmax(ov))
            r = R[k] / Lj.dot(R[k])
            r0 = sx.eta(tx).dot(r) / omega[k]
            Rx = State(r0, r)
        return float(self.overlap(Li, Rx, tx - res0.t))

    def coupling_fd(self, res0: Result, i: int, j: int, h1, B1, delta=2e-3):
        """Central differences with one Richardson step: error O(delta^4)."""
        O = {s: self.overlap_at(res0, i, j, s * delta, h1, B1) for s in (-2, -1, 1, 2)}
        return (8.0 * (O[1] - O[-1]) - (O[2] - O[-2])) / (12.0 * delta)
