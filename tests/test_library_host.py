"""Host-side checks of the CUDA library (no GPU needed).

* the shared library loads and exports every function include/ccsd.h declares;
* the tensor programs the library runs (residual and derivative programs,
  as described by ccsd_describe_program) reproduce the oracle when executed
  by a numpy interpreter: this checks the library's residual equations and its
  forward/reverse derivative transforms without a device.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from paper_2301_13264_gb300 import binding
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes
from ir_interp import Interp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(binding.LIB_PATH):
        from paper_2301_13264_gb300 import build
        build.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ccsd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_]+)\s*\([^;{]*\)\s*;", text)
    return sorted(set(n for n in names if n.startswith(("ccsd_", "eom_"))))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "ccsd_create" in names and "ccsd_derivative_coupling" in names and "eom_solve_left" in names
    for n in names:
        assert hasattr(L, n), n
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_strerror_and_defaults(L):
    assert binding.lib().ccsd_strerror(binding.ERR_COMPLEX_ROOT).decode() == "complex EOM root"
    opt = binding.ccsd_default_options()
    assert opt.precision == binding.PREC_FP64 and opt.diis_dim == 8 and opt.relax_orbitals == 0


def test_create_rejects_bad_arguments(L):
    H = make_hamiltonian(2, 3, 4, seed=0)
    with pytest.raises(binding.CCSDError) as e:
        binding.ccsd_create(H.eps, H.h, H.B, 0, 3, 4)
    assert e.value.status == binding.ERR_ARG
    opt = binding.ccsd_default_options(relax_orbitals=2)  # 0 or 1 only
    with pytest.raises(binding.CCSDError) as e:
        binding.ccsd_create(H.eps, H.h, H.B, 2, 3, 4, opt)
    assert e.value.status == binding.ERR_ARG
    opt = binding.ccsd_default_options(precision=3)  # FP64, MIXED or FP64_TC only
    with pytest.raises(binding.CCSDError) as e:
        binding.ccsd_create(H.eps, H.h, H.B, 2, 3, 4, opt)
    assert e.value.status == binding.ERR_ARG
    with pytest.raises(TypeError):
        binding.ccsd_default_options(no_such_option=1)


def test_fp64_tc_defaults_and_gemm_arguments(L):
    opt = binding.ccsd_default_options()
    assert opt.fp64_tc == 1
    A, Bm = np.ones((3, 4)), np.ones((2, 4))
    # checked before any device work: unknown form, beta outside {0, 1} on the tensor-core
    # forms, split counts other than 2 and 3, mismatched K
    for kw in (dict(form=7), dict(form=binding.GEMM_FP64_TC, beta=0.5), dict(form=binding.GEMM_SPLIT, splits=4)):
        form = kw.pop("form")
        with pytest.raises(binding.CCSDError) as e:
            binding.ccsd_gemm(form, A, Bm, C=np.zeros((3, 2)), **kw)
        assert e.value.status == binding.ERR_ARG
    with pytest.raises(ValueError):
        binding.ccsd_gemm(binding.GEMM_FP64, A, np.ones((2, 5)))


@pytest.fixture(scope="module")
def programs(L):
    return {w: binding.ccsd_describe_program(w) for w in ("fwd", "jvp", "vjp", "hvp", "dens1", "dens0")}


def _pg(g2, o, v):
    return cc.packed_grad(torch.zeros(o, v, dtype=torch.float64), torch.as_tensor(g2))[1].numpy()


@pytest.mark.parametrize("o,v,naux", [(2, 4, 6), (3, 5, 7), (1, 3, 2)])
def test_library_programs_match_oracle(programs, o, v, naux):
    H = make_hamiltonian(o, v, naux, seed=3)
    X1, X2 = random_amplitudes(o, v, 5, scale=0.1, nvec=8)
    t1, t2 = X1[0], X2[0]
    T = cc.as_t
    h, B = T(H.h), T(H.B)
    nv = 2
    I = Interp(o, v, naux, nv)
    I.arr.update(t1=t1.copy(), t2=t2.copy(), h=H.h.copy(), B=H.B.copy(), ones_o=np.ones(o))
    I.run(programs["fwd"])
    c1, c2, ce = cc.residual(T(t1), T(t2), h, B, o)
    assert np.abs(I.arr["O1"] - c1.numpy()).max() < 1e-13
    assert np.abs(I.arr["O2"] - c2.numpy()).max() < 1e-13
    assert abs(float(I.arr["E"]) - float(ce)) < 1e-12
    # A R for a block of two directions
    R1, R2 = X1[1:3], X2[1:3]
    I.arr.update(zR1=R1.copy(), zR2=R2.copy())
    I.run(programs["jvp"])
    for k in range(nv):
        a1, a2 = cc.jacobian_right(T(t1), T(t2), T(R1[k]), T(R2[k]), h, B, o)
        assert np.abs(I.arr["Jz(O1)"][k] - a1.numpy()).max() < 1e-13
        assert np.abs(I.arr["Jz(O2)"][k] - a2.numpy()).max() < 1e-13
    # L^T A (and eta in the second slot)
    w = cc.pair_weight(o, v).numpy()
    L1, L2 = X1[3:5], X2[3:5]
    I.arr.update(zL1=L1.copy(), zL2=w * L2, zLE=np.array([0.0, 1.0]))
    I.run(programs["vjp"])
    for k in range(nv):
        a1, a2 = cc.jacobian_left(T(t1), T(t2), T(L1[k]), T(L2[k]), h, B, o)
        if k == 1:
            e1, e2 = cc.eta(T(t1), T(t2), h, B, o)
            a1, a2 = a1 + e1, a2 + e2
        assert np.abs(I.arr["Vz(t1)"][k] - a1.numpy()).max() < 1e-13
        assert np.abs(_pg(I.arr["Vz(t2)"][k], o, v) - a2.numpy()).max() < 1e-13
    # F-matrix with energy part
    g1, g2, r1, r2 = X1[5], X2[5], X1[6], X2[6]
    I.arr.update(hG1=g1, hG2=w * g2, hG0=np.array(0.7), hR1=r1, hR2=r2)
    I.run(programs["hvp"])
    a1, a2 = cc.lagrangian_hessian_right(T(t1), T(t2), 0.7, T(g1), T(g2), T(r1), T(r2), h, B, o)
    assert np.abs(I.arr["H1(V1(t1))"] - a1.numpy()).max() < 1e-14
    assert np.abs(_pg(I.arr["H1(V1(t2))"], o, v) - a2.numpy()).max() < 1e-14
    # densities contracted with the perturbation direction
    z1, z2 = X1[7], X2[7]
    I.arr.update(dZ1=z1, dZ2=w * z2, dG1=g1, dG2=w * g2, dG0=np.array(0.7), dR1=r1, dR2=r2)
    I.run(programs["dens1"])
    F = (I.arr["VD(h)"] * H.h1).sum() + (I.arr["VD(B)"] * H.B1).sum()
    ox1, ox2, _ = cc.hamiltonian_derivative_residual(T(t1), T(t2), h, B, T(H.h1), T(H.B1), o)
    x1, x2, xe = cc.hamiltonian_derivative_jacobian(T(t1), T(t2), T(r1), T(r2), h, B, T(H.h1), T(H.B1), o)
    ref = float(cc.pdot(T(z1), T(z2), ox1, ox2) + 0.7 * xe + cc.pdot(T(g1), T(g2), x1, x2))
    assert abs(F - ref) < 1e-13 * max(1.0, abs(ref))
    I.arr.update(eZ1=z1, eZ2=w * z2, eE=np.array(0.3))
    I.run(programs["dens0"])
    F = (I.arr["VE(h)"] * H.h1).sum() + (I.arr["VE(B)"] * H.B1).sum()
    _, _, ex = cc.hamiltonian_derivative_residual(T(t1), T(t2), h, B, T(H.h1), T(H.B1), o)
    assert abs(F - float(cc.pdot(T(z1), T(z2), ox1, ox2)) - 0.3 * float(ex)) < 1e-13


@pytest.mark.parametrize("o,v,naux", [(2, 4, 6), (3, 5, 9)])
def test_orbital_programs_match_oracle(L, o, v, naux):
    """The library's Hartree-Fock programs (Fock ov block, A^HF x, the adjoint of the
    rotation map, the kappa-bar densities, the integral rotation) executed by the
    interpreter against the oracle's definitions."""
    from oracle import relaxed as rx
    H = make_hamiltonian(o, v, naux, seed=5)
    rng = np.random.default_rng(9)
    n = o + v
    base = dict(h=H.h.copy(), B=H.B.copy(), ones_o=np.ones(o))

    def run(which, **arrs):
        I = Interp(o, v, naux)
        I.arr.update(base)
        I.arr.update(arrs)
        I.run(binding.ccsd_describe_program(which))
        return I.arr

    F = rx.fock(H.h, H.B, o)[:o, o:].numpy()
    assert np.abs(run("hf_fock")["Fov"] - F).max() < 1e-13
    x = rng.normal(size=(o, v))
    A = rx.hf_hessian(H.h, H.B, o).numpy()
    assert np.abs(run("hf_A", kx=x)["HA(Fov)"] - (A @ x.reshape(-1)).reshape(o, v)).max() < 1e-12
    # adjoint of the rotation map: <x-bar, x> = <D, dh(x)> + <Z, dB(x)>
    D, Z = rng.normal(size=(n, n)), rng.normal(size=(naux, n, n))
    xbar = run("hf_rotT", rotT_D=D, rotT_Z=Z)["RT(kx)"]
    K = rx.kappa_matrix(x, o, n).numpy()
    dh = K.T @ H.h + H.h @ K
    dB = np.einsum("rp,Jrq->Jpq", K, H.B) + np.einsum("Jpr,rq->Jpq", H.B, K)
    assert abs((xbar * x).sum() - (D * dh).sum() - (Z * dB).sum()) < 1e-11
    # kappa-bar densities: <kH, h1> + <kB, B1> = kbar . dF_ov along (h1, B1)
    kb = rng.normal(size=(o, v))
    out = run("hf_kdens", kbar=kb)
    _, dF = torch.func.jvp(lambda hh, BB: rx.fock(hh, BB, o)[:o, o:], (cc.as_t(H.h), cc.as_t(H.B)),
                           (cc.as_t(H.h1), cc.as_t(H.B1)))
    lhs = (out["KD(h)"] * H.h1).sum() + (out["KD(B)"] * H.B1).sum()
    assert abs(lhs - float((cc.as_t(kb) * dF).sum())) < 1e-12
    U = torch.linalg.matrix_exp(rx.kappa_matrix(x * 0.1, o, n)).numpy()
    out = run("hf_rotate", U=U)
    hr, Br = rx.rotate(H.h, H.B, U)
    assert np.abs(out["h_rot"] - hr.numpy()).max() < 1e-13 and np.abs(out["B_rot"] - Br.numpy()).max() < 1e-13
