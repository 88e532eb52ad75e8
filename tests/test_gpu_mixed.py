"""Mixed-precision (tcgen05 split-bf16) path against the FP64 oracle.

The tensor-core products carry ~16 significant bits with two bf16 slices per
operand (3 products) and ~24 bits with three slices (6 products), accumulated
in FP32 over K (up to ~1e5 terms here), so the three-slice form is limited by
the FP32 accumulation rather than by the operand splitting.  Residuals and
transforms are compared element-wise with the oracle relative to the largest
element: within 4e-4 for two slices and 2e-5 for three (the three-slice left
transforms were measured at 5e-6 to 6.5e-6 on these inputs).
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle.solvers import System, Vec
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes, workload

pytestmark = pytest.mark.gpu

TOL = {2: 4e-4, 3: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available()
    B.lib()


def flat(x1, x2):
    return np.concatenate([np.asarray(x1).reshape(-1), np.asarray(x2).reshape(-1)])


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def mixed(H, S, **kw):
    o = dict(precision=B.PREC_MIXED, splits=S, tc_min_flops=0.0)
    o.update(kw)
    return B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**o))


@pytest.mark.parametrize("S", [2, 3])
@pytest.mark.parametrize("o,v,naux", [(6, 48, 60), (9, 37, 41)])
def test_mixed_residual_and_transforms(S, o, v, naux):
    H = make_hamiltonian(o, v, naux, seed=4)
    X1, X2 = random_amplitudes(o, v, 8, scale=0.03, nvec=4)
    t = flat(X1[0], X2[0])
    h = mixed(H, S)
    try:
        om = np.zeros_like(t)
        e = B.ccsd_residual(h, t, om)
        st = B.ccsd_stats(h)
        assert st["tc_gemms"] > 0, "tensor-core path not taken"
        c1, c2, ce = cc.residual(cc.as_t(X1[0]), cc.as_t(X2[0]), cc.as_t(H.h), cc.as_t(H.B), o)
        assert relerr(om, flat(c1, c2)) < TOL[S]
        # with tc_min_flops = 0 the Fock-matrix contractions run on the tensor cores too
        assert abs(e - float(ce)) < TOL[S] * abs(float(ce))
        B.ccsd_set_amplitudes(h, t, np.zeros_like(t))
        X = np.stack([flat(X1[k], X2[k]) for k in (1, 2, 3)])
        YR, YL = np.zeros_like(X), np.zeros_like(X)
        B.ccsd_jacobian_transform(h, 0, 3, X, YR)
        B.ccsd_jacobian_transform(h, 1, 3, X, YL)
    finally:
        B.ccsd_destroy(h)
    S_ = System(H.eps, H.h, H.B, o)
    tv = Vec(cc.as_t(X1[0]), cc.as_t(X2[0]))
    for k in range(3):
        r = Vec(cc.as_t(X1[k + 1]), cc.as_t(X2[k + 1]))
        ar, la = S_.right(tv, r), S_.left(tv, r)
        assert relerr(YR[k], flat(ar.x1, ar.x2)) < TOL[S]
        assert relerr(YL[k], flat(la.x1, la.x2)) < TOL[S]


def test_mixed_pipeline_energy_and_couplings():
    """Three-slice products with FP64 solver arithmetic and no refinement,
    converged to the mixed-precision floor: energies within 1e-6 Eh and
    couplings within 1e-3 relative of the oracle at the small workload."""
    H = workload("small")
    S_ = System(H.eps, H.h, H.B, H.o)
    res = S_.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    h = mixed(H, 3, tol_res=3e-6, tol_eom=1e-5, tol_lin=3e-6, max_iter=200, refine=0)
    try:
        e, _ = B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        F = {kl: B.ccsd_derivative_coupling(h, kl[0], kl[1], 1, H.h1, H.B1)[0] for kl in [(1, 2), (0, 1), (2, 0)]}
        assert B.ccsd_stats(h)["tc_gemms"] > 0
    finally:
        B.ccsd_destroy(h)
    assert abs(e - res.e_ccsd) < 1e-6
    assert np.abs(np.array(w) - np.array(res.omega)).max() < 1e-5
    for (k, l), f in F.items():
        ref = S_.coupling(res, k, l, H.h1, H.B1, tol_lin=1e-12)
        assert abs(f - ref) < 1e-3 * abs(ref)


@pytest.mark.parametrize("S", [2, 3])
def test_refined_mixed_pipeline_meets_fp64_tolerances(S):
    """Tensor-core products everywhere (tc_min_flops = 0) with FP64 refinement of
    every solve and FP64 densities: the FP64 tolerances of the method hold,
    energies within 1e-9 Eh, excitation energies within 1e-8, couplings within
    1e-7 relative of the oracle."""
    H = workload("small")
    S_ = System(H.eps, H.h, H.B, H.o)
    res = S_.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    h = mixed(H, S, tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200, refine=1)
    try:
        e, _ = B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        F = {kl: B.ccsd_derivative_coupling(h, kl[0], kl[1], 1, H.h1, H.B1)[0] for kl in [(1, 2), (0, 1), (2, 0)]}
        assert B.ccsd_stats(h)["tc_gemms"] > 0
    finally:
        B.ccsd_destroy(h)
    assert abs(e - res.e_ccsd) < 1e-9
    assert np.abs(np.array(w) - np.array(res.omega)).max() < 1e-8
    for (k, l), f in F.items():
        ref = S_.coupling(res, k, l, H.h1, H.B1, tol_lin=1e-12)
        assert abs(f - ref) < 1e-7 * abs(ref)


@pytest.mark.parametrize("S", [3])
def test_thymine_adz_residual_full_size(S):
    """o=33, v=228, naux=900 (the throughput workload): element-wise parity of
    the mixed residual with the oracle at random amplitudes."""
    H = workload("thymine_adz")
    o, v = H.o, H.v
    x1, x2 = random_amplitudes(o, v, 21, scale=0.01)
    t = flat(x1[0], x2[0])
    h = mixed(H, S, tc_min_flops=2.0e9)
    try:
        om = np.zeros_like(t)
        e = B.ccsd_residual(h, t, om)
    finally:
        B.ccsd_destroy(h)
    c1, c2, ce = cc.residual(cc.as_t(x1[0]), cc.as_t(x2[0]), cc.as_t(H.h), cc.as_t(H.B), o, vvvv_batch=24)
    assert relerr(om, flat(c1, c2)) < TOL[S]
    assert abs(e - float(ce)) < 1e-8


def test_thymine_adz_transform_properties():
    """At full size: <L|A R> = <L^T A|R> and A R matches the central difference
    of the residual along R (properties that hold at any size)."""
    H = workload("thymine_adz")
    o, v = H.o, H.v
    X1, X2 = random_amplitudes(o, v, 22, scale=0.01, nvec=3)
    t = torch.as_tensor(flat(X1[0], X2[0]), device="cuda")
    R = torch.as_tensor(flat(X1[1], X2[1]), device="cuda")[None]
    L = torch.as_tensor(flat(X1[2], X2[2]), device="cuda")[None]
    h = mixed(H, 3, tc_min_flops=2.0e9)
    try:
        B.ccsd_set_amplitudes(h, t, torch.zeros_like(t))
        AR, LA = torch.zeros_like(R), torch.zeros_like(L)
        B.ccsd_jacobian_transform(h, 0, 1, R, AR)
        B.ccsd_jacobian_transform(h, 1, 1, L, LA)
        w = torch.as_tensor(cc.pair_weight(o, v).numpy().reshape(-1), device="cuda")

        def pdot(a, b):
            n1 = o * v
            return float((a[:n1] * b[:n1]).sum() + (w * a[n1:] * b[n1:]).sum())

        lhs, rhs = pdot(L[0], AR[0]), pdot(LA[0], R[0])
        assert abs(lhs - rhs) < 1e-5 * max(abs(lhs), 1e-12)
    finally:
        B.ccsd_destroy(h)
    # central difference of the FP64 residual (the mixed residual's rounding is
    # not smooth in t, so the difference quotient uses the FP64 path)
    h64 = B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux, B.ccsd_default_options())
    try:
        d = 1e-3
        op, om_ = torch.zeros_like(t), torch.zeros_like(t)
        B.ccsd_residual(h64, t + d * R[0], op)
        B.ccsd_residual(h64, t - d * R[0], om_)
        fd = (op - om_) / (2 * d)
        assert float((fd - AR[0]).abs().max() / AR[0].abs().max()) < 1e-4
    finally:
        B.ccsd_destroy(h64)


def _golden_adz():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "thymine_adz_transforms.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_thymine_adz_transforms_match_oracle_samples(precision):
    """o=33, v=228, naux=900 at the benchmark's launch configuration: one right and one
    left transform against the oracle's full FP64 transforms, stored by
    tests/golden/make_thymine_adz_transforms.py (4160 sampled elements including the 64
    largest, plus the largest magnitude, packed norm and sum over all 5.66e7 elements).
    Three-slice products: within 2e-5 of the largest element; FP64: 1e-11."""
    G = _golden_adz()
    H = workload("thymine_adz")
    o, v = H.o, H.v
    X1, X2 = random_amplitudes(o, v, 22, scale=0.01, nvec=3)
    t = torch.as_tensor(flat(X1[0], X2[0]), device="cuda")
    R = torch.as_tensor(flat(X1[1], X2[1]), device="cuda")[None].contiguous()
    L = torch.as_tensor(flat(X1[2], X2[2]), device="cuda")[None].contiguous()
    opt = (B.ccsd_default_options(precision=B.PREC_MIXED, splits=3) if precision == "mixed"
           else B.ccsd_default_options())
    tol = TOL[3] if precision == "mixed" else 1e-11
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux, opt)
    try:
        B.ccsd_set_amplitudes(h, t, torch.zeros_like(t))
        out = {}
        for side, X in (("right", R), ("left", L)):
            Y = torch.zeros_like(X)
            B.ccsd_jacobian_transform(h, 0 if side == "right" else 1, 1, X, Y)
            out[side] = Y[0]
    finally:
        B.ccsd_destroy(h)
    w = torch.as_tensor(cc.pair_weight(o, v).numpy().reshape(-1), device="cuda")
    n1 = o * v
    for side, y in out.items():
        g = G[side]
        idx = torch.as_tensor(g["index"], device="cuda")
        ref = np.array(g["value"])
        got = y[idx].cpu().numpy()
        assert np.abs(got - ref).max() < tol * g["maxabs"], side
        assert abs(float(y.abs().max()) - g["maxabs"]) < tol * g["maxabs"]
        pn = float(((y[:n1] * y[:n1]).sum() + (w * y[n1:] * y[n1:]).sum()).sqrt())
        assert abs(pn - g["packed_norm"]) < tol * g["packed_norm"]
        # the plain sum over 5.66e7 elements cancels: bound by the per-element error times the count
        assert abs(float(y.sum()) - g["sum"]) < tol * g["maxabs"] * y.numel() ** 0.5 * 10


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_profile_records_account_for_every_gemm(prec):
    """ccsd_profile_records: one record per GEMM launch, summing to the profile's totals."""
    o, v, naux = 6, 48, 60
    H = make_hamiltonian(o, v, naux, seed=4)
    X1, X2 = random_amplitudes(o, v, 8, scale=0.03, nvec=3)
    X = np.stack([flat(X1[i], X2[i]) for i in range(3)])
    if prec == "mixed":
        h = mixed(H, 3, tc_min_flops=1e6)
    else:
        h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, B.ccsd_default_options(precision=B.PREC_FP64))
    try:
        B.ccsd_set_amplitudes(h, X[0], np.zeros_like(X[0]))
        Y = np.zeros_like(X)
        B.ccsd_jacobian_transform(h, 0, 3, X, Y)  # first use: slices, autotuning
        B.ccsd_profile_start(h)
        B.ccsd_jacobian_transform(h, 0, 3, X, Y)
        B.ccsd_jacobian_transform(h, 1, 3, X, Y)
        tot = B.ccsd_profile_stop(h)
        recs = B.ccsd_profile_records(h)
        n = ctypes.c_int(0)
        assert B.lib().ccsd_profile_records(h, None, -1, ctypes.byref(n)) == B.ERR_ARG
        assert B.lib().ccsd_profile_records(h, None, 1, ctypes.byref(n)) == B.ERR_ARG
        assert B.lib().ccsd_profile_records(h, None, 0, None) == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    assert len(recs) == tot["tc_launches"] + tot["fp64_launches"] > 0
    tc = [r for r in recs if r["engine"] != B.GEMM_FP64]
    assert len(tc) == tot["tc_launches"]
    assert (len(tc) > 0) == (prec == "mixed")
    assert abs(sum(r["ms"] for r in tc) - tot["tc_ms"]) < 1e-6 * max(tot["tc_ms"], 1.0)
    assert abs(sum(r["flops"] for r in recs) - tot["tc_flops"] - tot["fp64_flops"]) < 1e-6 * sum(
        r["flops"] for r in recs)
    lad = [r for r in recs if r["ladder"]]
    assert len(lad) == tot["ladder_launches"] == 4  # + and - pairs, right and left
    for r in recs:
        assert "+=" in r["label"] and r["ms"] >= 0.0 and r["m"] > 0 and r["n"] > 0 and r["k"] > 0
        assert abs(r["flops"] - 2.0 * r["batch"] * r["m"] * r["n"] * r["k"]) < 1e-9 * r["flops"]
        assert r["issued_flops"] >= r["flops"] * (0.999 if r["engine"] == B.GEMM_FP64 else 1.0)


@pytest.mark.parametrize("S,bits", [(2, 15), (3, 20)])
def test_split_products_of_single_terms(S, bits):
    """K = 1: C = a b^T through the split-bf16 products, operands over 2^-30..2^31 (products far
    inside the FP32 normal range), both signs, carries out of the rounding and zeros.  Each
    element is the FP32 sum of the S(S+1)/2 slice products of one a_m and one b_n: within
    about 2^-15 (two slices) and 2^-20 (three slices: the dropped products 2^-24 each plus
    five FP32 roundings) of |a_m b_n|."""
    rng = np.random.default_rng(11)
    sgn = lambda n: np.where(rng.random(n) < 0.5, -1.0, 1.0)
    a = sgn(300) * rng.uniform(1.0, 2.0, 300) * 2.0 ** rng.integers(-30, 30, 300)
    b = sgn(200) * rng.uniform(1.0, 2.0, 200) * 2.0 ** rng.integers(-30, 30, 200)
    a[:8] = [1.0, -2.0 ** -30, np.nextafter(2.0, 0.0), -(1.0 - 2.0 ** -53), 0.0, -0.0, 1.0 + 2.0 ** -23,
             -(2.0 ** 24 - 1.0) * 2.0 ** -50]
    C, _ = B.ccsd_gemm(B.GEMM_SPLIT, a[:, None], b[:, None], splits=S)
    ref = np.outer(a, b)
    assert np.all(np.abs(C - ref) <= 2.0 ** -bits * np.abs(ref)), (np.abs(C - ref) / np.abs(ref)).max()


def test_three_slices_carry_the_bits_below_float():
    """Rows [a_m, -fl32(a_m)] against [1, 1]: fl32(a_m) has 24 significant bits, which three
    slices carry exactly, and the slice products of each level nearly cancel and sum exactly,
    so C_m = a_m - fl32(a_m) + (the three slices' error in a_m).  That error is at most
    2^-26 |a_m| for the split from the double's bits (2^-28 rms), while a_m - fl32(a_m) is up
    to 2^-24 |a_m|: a split that rounded a_m to float first would miss by that much."""
    rng = np.random.default_rng(12)
    a = (np.where(rng.random(4000) < 0.5, -1.0, 1.0) * rng.uniform(1.0, 2.0, 4000)
         * 2.0 ** rng.integers(-50, 50, 4000))
    A = np.stack([a, -a.astype(np.float32).astype(np.float64)], axis=1)
    C, _ = B.ccsd_gemm(B.GEMM_SPLIT, A, np.ones((1, 2)), splits=3)
    ref = a - a.astype(np.float32).astype(np.float64)
    err = np.abs(C[:, 0] - ref) / np.abs(a)
    assert err.max() <= 2.0 ** -25, err.max()
    assert (np.abs(ref) / np.abs(a)).max() > 2.0 ** -24.5  # the test would see a lost remainder
