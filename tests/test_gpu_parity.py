"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

FP64 path: residuals and transforms must agree with the oracle to roundoff
(1e-11 relative of the largest element); solved energies within 1e-8 Eh,
excitation energies within 1e-8 and derivative couplings within 1e-7
relative (the plain-FP64 tolerances of the method's accuracy target).
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle.fockspace import CCBruteForce
from oracle.solvers import System, Vec
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes, workload

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.lib()


def flat(x1, x2):
    return np.concatenate([np.asarray(x1).reshape(-1), np.asarray(x2).reshape(-1)])


def split(x, o, v):
    return x[: o * v].reshape(o, v), x[o * v:].reshape(o, o, v, v)


class Handle:
    def __init__(self, H, **opt):
        self.H = H
        self.h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**opt))
        self.dim = B.vector_dim(H.o, H.v)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        B.ccsd_destroy(self.h)


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("o,v,naux", [(1, 5, 6), (2, 4, 6), (3, 7, 10), (5, 20, 75)])
def test_residual_matches_oracle(o, v, naux):
    H = make_hamiltonian(o, v, naux, seed=11)
    x1, x2 = random_amplitudes(o, v, 2, scale=0.05)
    t = flat(x1[0], x2[0])
    om = np.zeros_like(t)
    with Handle(H) as hd:
        e = B.ccsd_residual(hd.h, t, om)
    c1, c2, ce = cc.residual(cc.as_t(x1[0]), cc.as_t(x2[0]), cc.as_t(H.h), cc.as_t(H.B), o)
    assert relerr(om, flat(c1, c2)) < 1e-12
    assert abs(e - float(ce)) < 1e-11


@pytest.mark.parametrize("o,v,naux,nvec", [(2, 4, 6, 3), (3, 7, 10, 5), (5, 20, 75, 9)])
def test_transforms_match_oracle(o, v, naux, nvec):
    H = make_hamiltonian(o, v, naux, seed=7)
    S = System(H.eps, H.h, H.B, o)
    with Handle(H, **TIGHT) as hd:
        e, _ = B.ccsd_solve_ground(hd.h)
        t = np.zeros(hd.dim)
        B.ccsd_get_amplitudes(hd.h, t)
        X1, X2 = random_amplitudes(o, v, 3, scale=0.1, nvec=nvec)
        X = np.stack([flat(X1[k], X2[k]) for k in range(nvec)])
        # device in/out for the right transform, host for the left one
        Xd = torch.as_tensor(X, device="cuda")
        Yd = torch.zeros_like(Xd)
        B.ccsd_jacobian_transform(hd.h, 0, nvec, Xd, Yd)
        YR = Yd.cpu().numpy()
        YL = np.zeros_like(X)
        B.ccsd_jacobian_transform(hd.h, 1, nvec, X, YL)
    tv = Vec(*map(cc.as_t, split(t, o, v)))
    _, e_or = S.residual(tv)
    assert abs(e - e_or) < 1e-10
    for k in range(nvec):
        r = Vec(cc.as_t(X1[k]), cc.as_t(X2[k]))
        ar = S.right(tv, r)
        la = S.left(tv, r)
        assert relerr(YR[k], flat(ar.x1, ar.x2)) < 1e-11
        assert relerr(YL[k], flat(la.x1, la.x2)) < 1e-11


@pytest.fixture(scope="module")
def small_pipeline():
    H = workload("small")
    S = System(H.eps, H.h, H.B, H.o)
    res = S.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    return H, S, res


def test_ground_and_eom_match_oracle(small_pipeline):
    H, S, res = small_pipeline
    o, v = H.o, H.v
    with Handle(H, **TIGHT) as hd:
        e, it = B.ccsd_solve_ground(hd.h)
        w, _ = B.eom_solve_right(hd.h, 2)
        wl, _ = B.eom_solve_left(hd.h, 2)
        t, lam = np.zeros(hd.dim), np.zeros(hd.dim)
        B.ccsd_get_amplitudes(hd.h, t, lam)
        R, L = np.zeros((2, hd.dim)), np.zeros((2, hd.dim))
        r0 = B.ccsd_get_states(hd.h, 2, R, L)
    assert abs(e - res.e_ccsd) < 1e-9
    assert np.abs(np.array(w) - np.array(res.omega)).max() < 1e-9
    assert np.abs(np.array(wl) - np.array(res.omega)).max() < 1e-9
    assert relerr(t, flat(res.t.x1, res.t.x2)) < 1e-8
    assert relerr(lam, flat(res.lam.x1, res.lam.x2)) < 1e-7
    for k in range(2):
        assert relerr(R[k], flat(res.right[k].vec.x1, res.right[k].vec.x2)) < 1e-6
        assert relerr(L[k], flat(res.left[k].vec.x1, res.left[k].vec.x2)) < 1e-6
        assert abs(r0[k] - res.right[k].c0) < 1e-8 * max(1.0, abs(res.right[k].c0))


@pytest.mark.parametrize("k,l", [(1, 2), (2, 1), (0, 1), (1, 0), (0, 2), (2, 0)])
def test_couplings_match_oracle(small_pipeline, k, l):
    H, S, res = small_pipeline
    ref = S.coupling(res, k, l, H.h1, H.B1, tol_lin=1e-12)
    with Handle(H, **TIGHT) as hd:
        B.ccsd_solve_ground(hd.h)
        B.eom_solve_right(hd.h, 2)
        B.eom_solve_left(hd.h, 2)
        F = B.ccsd_derivative_coupling(hd.h, k, l, 1, H.h1, H.B1)
    assert abs(F[0] - ref) < 1e-7 * abs(ref)


def test_two_electron_pipeline_is_exact():
    o, v = 1, 5
    H = make_hamiltonian(o, v, 6, seed=2)
    bf = CCBruteForce(H.h, H.B, o)
    w_fci, U = bf.fci()
    with Handle(H, **TIGHT) as hd:
        e, _ = B.ccsd_solve_ground(hd.h)
        w, _ = B.eom_solve_right(hd.h, 3)
    assert abs(e - w_fci[0]) < 1e-9
    assert np.abs(np.array(w) - (w_fci[1:4] - w_fci[0])).max() < 1e-8


def test_densities_give_coupling_in_several_directions(small_pipeline):
    H, S, res = small_pipeline
    n, naux = H.n, H.naux
    rng = np.random.default_rng(3)
    dh = np.stack([H.h1, 0.5 * (lambda m: m + m.T)(rng.normal(size=(n, n)))])
    dB = np.stack([H.B1, np.zeros_like(H.B1)])
    with Handle(H, **TIGHT) as hd:
        B.ccsd_solve_ground(hd.h)
        B.eom_solve_right(hd.h, 2)
        B.eom_solve_left(hd.h, 2)
        D = np.zeros((n, n))
        Z = np.zeros((naux, n, n))
        B.ccsd_coupling_densities(hd.h, 1, 2, D, Z)
        F = B.ccsd_derivative_coupling(hd.h, 1, 2, 2, torch.as_tensor(dh, device="cuda"),
                                       torch.as_tensor(dB, device="cuda"))
    assert abs(F[0] - ((D * dh[0]).sum() + (Z * dB[0]).sum())) < 1e-12
    ref = S.coupling(res, 1, 2, dh[1], dB[1], tol_lin=1e-12)
    assert abs(F[1] - ref) < 1e-7 * abs(ref)


def test_error_statuses():
    H = make_hamiltonian(2, 4, 6, seed=1)
    with Handle(H) as hd:
        with pytest.raises(B.CCSDError) as e:
            B.eom_solve_right(hd.h, 2)
        assert e.value.status == B.ERR_STATE
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_coupling_densities(hd.h, 1, 1, np.zeros((6, 6)))
        assert e.value.status == B.ERR_ARG
        B.ccsd_solve_ground(hd.h)
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_derivative_coupling(hd.h, 0, 3, 1, H.h1, H.B1)
        assert e.value.status in (B.ERR_ARG, B.ERR_STATE)
    bad = H.B.copy()
    bad[0, 0, 1] += 1e-3
    with pytest.raises(B.CCSDError) as e:
        B.ccsd_create(H.eps, H.h, bad, 2, 4, 6)
    assert e.value.status == B.ERR_ARG
    opt = B.ccsd_default_options(max_iter=1)
    with Handle(H, **{"max_iter": 1}) as hd:
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_solve_ground(hd.h)
        assert e.value.status == B.ERR_NOT_CONVERGED


def test_thymine_dz_residual_and_transforms_full_size():
    """Thymine/cc-pVDZ-shaped system (o=33, v=123, naux=550): the FP64 residual and a block of
    two right and left Jacobian transforms at given amplitudes, element-wise against the
    oracle (every FP64 GEMM shape of the transform programs at full size, the skinny
    nvec-wide ones included)."""
    H = workload("thymine_dz")
    o, v = H.o, H.v
    x1, x2 = random_amplitudes(o, v, 4, scale=0.01, nvec=3)
    t = flat(x1[0], x2[0])
    X = np.stack([flat(x1[k], x2[k]) * 10.0 for k in (1, 2)])
    om = np.zeros_like(t)
    YR, YL = np.zeros_like(X), np.zeros_like(X)
    with Handle(H) as hd:
        e = B.ccsd_residual(hd.h, t, om)
        B.ccsd_set_amplitudes(hd.h, t, np.zeros_like(t))
        B.ccsd_jacobian_transform(hd.h, 0, 2, X, YR)
        B.ccsd_jacobian_transform(hd.h, 1, 2, X, YL)
    c1, c2, ce = cc.residual(cc.as_t(x1[0]), cc.as_t(x2[0]), cc.as_t(H.h), cc.as_t(H.B), o)
    assert relerr(om, flat(c1, c2)) < 1e-11
    assert abs(e - float(ce)) < 1e-9
    S = System(H.eps, H.h, H.B, o, vvvv_batch=16)
    tv = Vec(cc.as_t(x1[0]), cc.as_t(x2[0]))
    for k, side in ((0, "right"), (1, "right"), (0, "left")):
        r = Vec(*map(cc.as_t, split(X[k], o, v)))
        ref = S.right(tv, r) if side == "right" else S.left(tv, r)
        got = (YR if side == "right" else YL)[k]
        assert relerr(got, flat(ref.x1, ref.x2)) < 1e-11, (k, side)
