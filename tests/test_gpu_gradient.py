"""State-energy gradients and the branching plane on the GPU against the oracle.

The oracle's gradients (energy Lagrangian: E + lambda.Omega, plus L_k.(A R_k) + zeta.Omega
for excited states) are pinned to full CI for two electrons and to finite differences of
E_k(x) (tests/test_oracle_gradient.py), its relaxed gradients to finite differences with
re-optimised Hartree-Fock orbitals, and its crossing-point direction to the full-CI one
(tests/test_oracle_meci.py).  Tolerances: the gradients are stationary in every multiplier,
so they carry the solver thresholds to second order: 1e-7 relative (plus 1e-10 absolute),
the coupling tolerance of the method.
"""
import numpy as np
import pytest
import torch

from oracle import meci
from oracle import relaxed as rx
from oracle.solvers import System
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, workload

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available()
    B.lib()


def close(a, b, rel=1e-7, ab=1e-10):
    return abs(a - b) <= rel * abs(b) + ab


@pytest.fixture(scope="module")
def small_oracle():
    H = workload("small")
    S = System(H.eps, H.h, H.B, H.o)
    res = S.run(2, tol=1e-12, tol_eom=1e-10, tol_lin=1e-12)
    # a second direction: another draw of the same generator's perturbation
    H2 = make_hamiltonian(H.o, H.v, H.naux, seed=7)
    dirs = [(H.h1, H.B1), (H2.h1, H2.B1)]
    g = {k: [S.energy_gradient(res, k, dh, dB, tol_lin=1e-12) for dh, dB in dirs] for k in range(3)}
    f12 = [S.coupling(res, 1, 2, dh, dB, tol_lin=1e-12) for dh, dB in dirs]
    E = [res.e_ccsd + w for w in res.omega]
    return H, dirs, g, f12, E


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_energy_gradients_match_oracle(small_oracle, form):
    H, dirs, g_ref, _, _ = small_oracle
    kw = dict(TIGHT)
    if form == "mixed":
        kw.update(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0, refine=1)
    dh = np.ascontiguousarray(np.stack([d[0] for d in dirs]))
    dB = np.ascontiguousarray(np.stack([d[1] for d in dirs]))
    h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**kw))
    try:
        B.ccsd_solve_ground(h)
        g0 = B.ccsd_energy_gradient(h, 0, 2, dh, dB)   # needs only the ground state
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        g = {k: B.ccsd_energy_gradient(h, k, 2, dh, dB) for k in (1, 2, 0)}
        # the densities themselves, contracted on the host, give the same numbers
        n = H.o + H.v
        D, Z = np.zeros((n, n)), np.zeros((H.naux, n, n))
        B.ccsd_gradient_densities(h, 1, D, Z)
        # a coupling in between leaves the gradient densities recomputable
        B.ccsd_derivative_coupling(h, 1, 2, 1, H.h1, H.B1)
        g1_again = B.ccsd_energy_gradient(h, 1, 1, H.h1, H.B1)[0]
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_energy_gradient(h, 3, 1, H.h1, H.B1)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    for d in range(2):
        assert close(g0[d], g_ref[0][d]), (d, g0[d], g_ref[0][d])
        for k in range(3):
            assert close(g[k][d], g_ref[k][d]), (k, d, g[k][d], g_ref[k][d])
    assert close(float((D * dh[0]).sum() + (Z * dB[0]).sum()), g_ref[1][0])
    assert close(g1_again, g_ref[1][0])
    # the excited-state gradients differ from the ground state's (the test is not trivial)
    assert abs(g_ref[1][0] - g_ref[0][0]) > 1e-4


def test_gradient_needs_states():
    H = make_hamiltonian(2, 4, 6, seed=1)
    h = B.ccsd_create(H.eps, H.h, H.B, 2, 4, 6, B.ccsd_default_options())
    try:
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_energy_gradient(h, 0, 1, H.h1, H.B1)
        assert err.value.status == B.ERR_STATE
        B.ccsd_solve_ground(h)
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_energy_gradient(h, 1, 1, H.h1, H.B1)
        assert err.value.status in (B.ERR_STATE, B.ERR_ARG)
    finally:
        B.ccsd_destroy(h)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_branching_plane_matches_oracle(small_oracle, form):
    """g = grad(E_2 - E_1), h = (E_2 - E_1) F_12 and the Bearpark-Robb-Schlegel direction
    G = P grad E_2 + 2 (E_2 - E_1) g/|g| over two directions, against the oracle's quantities
    combined by the oracle's crossing-point search step."""
    H, dirs, g_ref, f12, E = small_oracle
    kw = dict(TIGHT)
    if form == "mixed":
        kw.update(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0, refine=1)
    dh = np.ascontiguousarray(np.stack([d[0] for d in dirs]))
    dB = np.ascontiguousarray(np.stack([d[1] for d in dirs]))
    h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**kw))
    try:
        B.ccsd_solve_ground(h)
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        gv, hv, G = B.ccsd_branching_plane(h, 1, 2, 2, torch.as_tensor(dh, device="cuda"),
                                           torch.as_tensor(dB, device="cuda"))
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_branching_plane(h, 0, 1, 2, dh, dB)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    g1, g2, f = np.array(g_ref[1]), np.array(g_ref[2]), np.array(f12)
    G_ref = meci.bearpark_direction(E[0], E[1], g1, g2, f)
    scale = max(np.abs(G_ref).max(), np.abs(g2).max())
    assert np.abs(np.array(gv) - (g2 - g1)).max() < 1e-7 * np.abs(g2 - g1).max() + 1e-10
    assert np.abs(np.array(hv) - (E[1] - E[0]) * f).max() < 1e-7 * np.abs((E[1] - E[0]) * f).max() + 1e-10
    assert np.abs(np.array(G) - G_ref).max() < 1e-7 * scale + 1e-10


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_relaxed_energy_gradients_match_oracle(precision):
    """Hartree-Fock orbitals that follow x add kappa-bar_ai F^x_ai (no overlap term in
    k-eta); the orbital term is resolved well above the tolerance."""
    o, v, naux = 3, 8, 16
    H = make_hamiltonian(o, v, naux, seed=16, bscale=0.3)
    U, hr, Br, _ = B.ccsd_scf(H.eps, H.h, H.B, o, v, naux, tol=1e-13)
    h1, B1 = B.ccsd_rotate_integrals(U, H.h1, H.B1, o, v, naux)
    kw = dict(TIGHT)
    if precision == B.PREC_MIXED:
        kw.update(splits=3, tc_min_flops=0.0, refine=1)
    g, gu = {}, {}
    for relax in (1, 0):
        h = B.ccsd_create(H.eps, hr, Br, o, v, naux,
                          B.ccsd_default_options(precision=precision, relax_orbitals=relax, **kw))
        try:
            B.ccsd_solve_ground(h)
            B.eom_solve_right(h, 2)
            B.eom_solve_left(h, 2)
            for k in range(3):
                (g if relax else gu)[k] = B.ccsd_energy_gradient(h, k, 1, h1, B1)[0]
        finally:
            B.ccsd_destroy(h)
    _, Uo, ho, Bo = rx.scf(H.h, H.B, o)
    h1o, B1o = rx.rotate(H.h1, H.B1, Uo)
    S = System(H.eps, ho, Bo, o)
    res = S.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    for k in range(3):
        ref = rx.relaxed_energy_gradient(S, res, k, h1o, B1o, tol_lin=1e-12)
        assert close(g[k], ref), (k, g[k], ref)
        assert abs(g[k] - gu[k]) > 100 * abs(g[k] - ref)
