"""Closed-shell CCSD residual, energy and their derivatives (oracle, FP64 CPU).

Test infrastructure of the oracle; see the package docstring.

Conventions (Theory section, "Lagrangian"):
* orbitals: occupied i,j,k,l first, then virtual a,b,c,d; n = o + v;
* integrals: h_pq and g_pqrs = (pq|rs) = sum_P B^P_pq B^P_rs (Cholesky factors,
  as used by the paper's implementation);
* amplitudes: t1[i,a] = t_ai, t2[i,j,a,b] = t_aibj = t_ij^ab with t2[i,j,a,b] =
  t2[j,i,b,a]; T = sum t_ai E_ai + 1/2 sum t_aibj E_ai E_bj;
* residual Omega_mu = <mu~|exp(-T) H exp(T)|HF> in the biorthonormal basis,
  stored in the same unpacked layout (the packed coefficient of tau_aibj,
  ai >= bj, is stored at both [i,j,a,b] and [j,i,b,a]);
* inner product of two vectors is the packed one,
  <L|R> = sum_ai L_ai R_ai + sum_{ai >= bj} L_aibj R_aibj, see :func:`pdot`.

The residual is written in the T1-transformed form: with X = 1 - t1 and
Y = 1 + t1 (t1 placed in the virtual-occupied block), exp(-T1) H exp(T1) has
integrals h^ = X h Y and B^P^ = X B^P Y, and the remaining doubles equations
are the standard closed-shell CCSD terms over these dressed integrals.
The Jacobian A_mu,nu = <mu~|[Hbar, tau_nu]|HF> (Eq. for A) is the derivative of
Omega with respect to t_nu, and the F-matrix (Eq. for F) the second
derivative of the contracted residual; both are obtained here by automatic
differentiation of the residual, so that no separate transformation formulas
can disagree with it.
"""
from __future__ import annotations

import torch
from torch import einsum

F64 = torch.float64


def as_t(x):
    if isinstance(x, torch.Tensor):
        return x.to(F64)
    return torch.as_tensor(x, dtype=F64)


# ---------------------------------------------------------------------------
# packed metric helpers
# ---------------------------------------------------------------------------

def pair_weight(o: int, v: int) -> torch.Tensor:
    """w[i,j,a,b] = 1/2 for (ai) != (bj), 1 for (ai) == (bj).

    sum_{ai>=bj} L R = sum_all w L R for pair-symmetric tensors.
    """
    w = torch.full((o, o, v, v), 0.5, dtype=F64)
    for i in range(o):
        for a in range(v):
            w[i, i, a, a] = 1.0
    return w


def pdot(l1, l2, r1, r2) -> torch.Tensor:
    """Packed inner product sum_ai l_ai r_ai + sum_{ai>=bj} l_aibj r_aibj."""
    o, v = l1.shape
    w = pair_weight(o, v)
    return (l1 * r1).sum() + (w * l2 * r2).sum()


def packed_grad(g1, g2):
    """Convert d/d(unpacked storage) into d/d(packed coordinate).

    For ai != bj the packed coordinate t_aibj is stored twice, so its derivative
    is the sum of the two storage derivatives; the diagonal is stored once.
    Result is returned in unpacked, pair-symmetric storage.
    """
    o, v = g1.shape
    s = g2 + g2.permute(1, 0, 3, 2)
    idx_i = torch.arange(o)
    idx_a = torch.arange(v)
    s = s.clone()
    for i in range(o):
        s[i, i, idx_a, idx_a] = g2[i, i, idx_a, idx_a]
    return g1, s


def symmetrize_pairs(x2):
    return 0.5 * (x2 + x2.permute(1, 0, 3, 2))


# ---------------------------------------------------------------------------
# T1-transformed integrals, Fock matrix, residual and energy
# ---------------------------------------------------------------------------

def t1_matrices(t1, o: int, n: int):
    """X = 1 - t1 and Y = 1 + t1, with t1[a, i] placed in the (virtual, occupied) block."""
    v = n - o
    z_oo = torch.zeros((o, o), dtype=F64)
    z_on = torch.zeros((o, n), dtype=F64)
    z_vv = torch.zeros((v, v), dtype=F64)
    emb = torch.cat([z_on, torch.cat([t1.T, z_vv], dim=1)], dim=0)
    eye = torch.eye(n, dtype=F64)
    return eye - emb, eye + emb


def dressed(h, B, t1, o):
    """h^ = X h Y and B^P^ = X B^P Y."""
    n = h.shape[0]
    X, Y = t1_matrices(t1, o, n)
    return X @ h @ Y, torch.matmul(torch.matmul(X, B), Y)


def fock(hh, Bh, o):
    """F_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)] (closed-shell Fock matrix).

    The paper prints the two integral labels of this sum in the other order;
    the standard restricted Fock operator (Coulomb twice, exchange once) is the
    one that makes <HF|H|HF> = sum_i (h_ii + F_ii), which the determinant-space
    tests check.
    """
    d = einsum("Pkk->P", Bh[:, :o, :o])
    return hh + 2.0 * einsum("Ppq,P->pq", Bh, d) - einsum("Ppk,Pkq->pq", Bh[:, :, :o], Bh[:, :o, :])


def _g(Bh, s1, s2, s3, s4):
    return einsum("Ppq,Prs->pqrs", Bh[:, s1, s2], Bh[:, s3, s4])


def residual(t1, t2, h, B, o, vvvv_batch: int | None = None):
    """Closed-shell CCSD (Omega1[i,a], Omega2[i,j,a,b], E) over dressed integrals.

    Terms (with u_ij^ab = 2 t_ij^ab - t_ij^ba, L_pqrs = 2 g_pqrs - g_psrq and
    P the pair permutation (ai) <-> (bj)):

    Omega_ai  = F_ai + sum u_ki^cd g_adkc - sum u_kl^ac g_kilc + sum u_ik^ac F_kc
    Omega_aibj = g_aibj + sum t_ij^cd g_acbd + sum t_kl^ab (g_kilj + sum t_ij^cd g_kcld)
               + P[ -1/2 sum t_kj^bc C_kiac - sum t_ki^bc C_kjac
                    + 1/2 sum u_jk^bc D_aikc
                    + sum t_ij^ac (F_bc - sum u_kl^bd g_ldkc)
                    - sum t_ik^ab (F_kj + sum u_lj^cd g_kdlc) ]
    C_kiac = g_kiac - 1/2 sum t_li^ad g_kdlc,  D_aikc = L_aikc + 1/2 sum u_il^ad L_ldkc
    E = sum_i (h_ii + F_ii) + sum t_ij^ab L_iajb.
    All integrals and F are T1-dressed.
    """
    n = h.shape[0]
    v = n - o
    O, V = slice(0, o), slice(o, n)
    hh, Bh = dressed(h, B, t1, o)
    F = fock(hh, Bh, o)
    u = 2.0 * t2 - t2.permute(0, 1, 3, 2)

    # singles
    om1 = F[V, O].T.clone()
    om1 = om1 + einsum("kicd,adkc->ia", u, _g(Bh, V, V, O, V))
    om1 = om1 - einsum("klac,kilc->ia", u, _g(Bh, O, O, O, V))
    om1 = om1 + einsum("ikac,kc->ia", u, F[O, V])

    # doubles, before the pair permutation (symmetric pieces carry 1/2)
    g_ovov = _g(Bh, O, V, O, V)            # [k,c,l,d]  (undressed block)
    L_ovov = 2.0 * g_ovov - g_ovov.permute(0, 3, 2, 1)
    r = 0.5 * einsum("aibj->ijab", _g(Bh, V, O, V, O))
    if vvvv_batch is None:
        r = r + 0.5 * einsum("ijcd,acbd->ijab", t2, _g(Bh, V, V, V, V))
    else:
        parts = []
        for a0 in range(0, v, vvvv_batch):
            a1 = min(v, a0 + vvvv_batch)
            gblk = einsum("Pac,Pbd->acbd", Bh[:, o + a0:o + a1, V], Bh[:, V, V])
            parts.append(einsum("ijcd,acbd->ijab", t2, gblk))
        r = r + 0.5 * torch.cat(parts, dim=2)
    chi = einsum("kilj->kilj", _g(Bh, O, O, O, O)) + einsum("ijcd,kcld->kilj", t2, g_ovov)
    r = r + 0.5 * einsum("klab,kilj->ijab", t2, chi)
    C = einsum("kiac->kiac", _g(Bh, O, O, V, V)) - 0.5 * einsum("liad,kdlc->kiac", t2, g_ovov)
    r = r - 0.5 * einsum("kjbc,kiac->ijab", t2, C)
    r = r - einsum("kibc,kjac->ijab", t2, C)
    g_voov = _g(Bh, V, O, O, V)            # [a,i,k,c]
    g_vvoo = _g(Bh, V, V, O, O)            # [a,c,k,i]
    L_voov = 2.0 * g_voov - einsum("acki->aikc", g_vvoo)
    D = L_voov + 0.5 * einsum("ilad,ldkc->aikc", u, L_ovov)
    r = r + 0.5 * einsum("jkbc,aikc->ijab", u, D)
    Gvv = F[V, V] - einsum("klbd,ldkc->bc", u, g_ovov)
    r = r + einsum("ijac,bc->ijab", t2, Gvv)
    Goo = F[O, O] + einsum("ljcd,kdlc->kj", u, g_ovov)
    r = r - einsum("ikab,kj->ijab", t2, Goo)
    om2 = r + r.permute(1, 0, 3, 2)

    e = torch.diagonal(hh[O, O]).sum() + torch.diagonal(F[O, O]).sum() + einsum("ijab,iajb->", t2, L_ovov)
    return om1, om2, e


# ---------------------------------------------------------------------------
# derivatives
# ---------------------------------------------------------------------------

def _zeros_like_amps(o, v):
    return torch.zeros((o, v), dtype=F64), torch.zeros((o, o, v, v), dtype=F64)


def jacobian_right(t1, t2, r1, r2, h, B, o, **kw):
    """(A R)_mu = sum_nu dOmega_mu/dt_nu R_nu (directional derivative)."""
    f = lambda a, b: residual(a, b, h, B, o, **kw)[:2]
    _, (d1, d2) = torch.func.jvp(f, (t1, t2), (r1, r2))
    return d1, d2


def jacobian_left(t1, t2, l1, l2, h, B, o, **kw):
    """(L^T A)_nu = d/dt_nu <L|Omega(t)> in packed coordinates, stored unpacked."""
    w = pair_weight(o, t1.shape[1])
    f = lambda a, b: residual(a, b, h, B, o, **kw)[:2]
    _, vjp = torch.func.vjp(f, t1, t2)
    g1, g2 = vjp((l1, w * l2))
    return packed_grad(g1, g2)


def eta(t1, t2, h, B, o, **kw):
    """eta_nu = <HF|[Hbar, tau_nu]|HF> = dE/dt_nu (packed)."""
    f = lambda a, b: residual(a, b, h, B, o, **kw)[2]
    g1, g2 = torch.func.grad(f, argnums=(0, 1))(t1, t2)
    return packed_grad(g1, g2)


def lagrangian_hessian_right(t1, t2, g0, g1, g2, r1, r2, h, B, o, **kw):
    """sum_nu d^2 (g0 E + <g|Omega>)/dt_sigma dt_nu R_nu, packed in sigma.

    With g0 = 0 this is the F-matrix transformation (F(g) R)_sigma of the
    paper; g0 multiplies the second derivative of the energy, which is the
    <HF| part of <g| in <g|[[Hbar, tau_sigma], tau_nu]|HF>.
    """
    w = pair_weight(o, t1.shape[1])

    def scal(a, b):
        om1, om2, e = residual(a, b, h, B, o, **kw)
        return g0 * e + (g1 * om1).sum() + (w * g2 * om2).sum()

    grad = torch.func.grad(scal, argnums=(0, 1))
    _, (d1, d2) = torch.func.jvp(lambda a, b: grad(a, b), (t1, t2), (r1, r2))
    return packed_grad(d1, d2)


def hamiltonian_derivative_residual(t1, t2, h, B, h1, B1, o, **kw):
    """(Omega^x, E^x): derivative of residual and energy along h + x h1, B + x B1 at fixed t."""
    f = lambda hh, BB: residual(t1, t2, hh, BB, o, **kw)
    _, (d1, d2, de) = torch.func.jvp(f, (h, B), (h1, B1))
    return d1, d2, de


def hamiltonian_derivative_jacobian(t1, t2, r1, r2, h, B, h1, B1, o, **kw):
    """d/dx of (A R, eta^T R) at fixed t and R: <mu~|[Hbar^x, R]|HF> and <HF|[Hbar^x, R]|HF>."""
    def ar(hh, BB):
        f = lambda a, b: residual(a, b, hh, BB, o, **kw)
        _, (d1, d2, de) = torch.func.jvp(f, (t1, t2), (r1, r2))
        return d1, d2, de
    _, (x1, x2, xe) = torch.func.jvp(ar, (h, B), (h1, B1))
    return x1, x2, xe
