"""Orbital relaxation on the GPU against the oracle.

The library's Hartree-Fock orbitals (nearest ones, occupied-virtual rotation) and
rotated integrals equal the oracle's; a handle with relax_orbitals = 1 refuses
non-Hartree-Fock orbitals; and the relaxed couplings (kappa-bar from the
Hartree-Fock Hessian, the transition density and the condition densities) equal
the oracle's relaxed couplings, which are pinned to determinant-space finite
differences of the definition with re-optimised orbitals.
"""
import numpy as np
import pytest

from oracle import relaxed as rx
from oracle.solvers import System
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def test_scf_matches_oracle():
    o, v, naux = 3, 9, 20
    H = make_hamiltonian(o, v, naux, seed=11, bscale=0.3)
    U, hr, Br, it = B.ccsd_scf(H.eps, H.h, H.B, o, v, naux, tol=1e-13)
    kappa, Uo, ho, Bo = rx.scf(H.h, H.B, o)
    assert it >= 2 and float(kappa.abs().max()) > 1e-3
    assert np.abs(U - Uo.numpy()).max() < 1e-11
    assert np.abs(hr - ho.numpy()).max() < 1e-11
    assert np.abs(Br - Bo.numpy()).max() < 1e-11
    h1, B1 = B.ccsd_rotate_integrals(U, H.h1, H.B1, o, v, naux)
    h1o, B1o = rx.rotate(H.h1, H.B1, Uo)
    assert np.abs(h1 - h1o.numpy()).max() < 1e-12 and np.abs(B1 - B1o.numpy()).max() < 1e-12


def test_relaxed_mode_needs_hartree_fock_orbitals():
    o, v, naux = 2, 6, 12
    H = make_hamiltonian(o, v, naux, seed=12)
    opt = B.ccsd_default_options(relax_orbitals=1)
    with pytest.raises(B.CCSDError) as e:
        B.ccsd_create(H.eps, H.h, H.B, o, v, naux, opt)
    assert e.value.status == B.ERR_NOT_HF
    _, hr, Br, _ = B.ccsd_scf(H.eps, H.h, H.B, o, v, naux)
    h = B.ccsd_create(H.eps, hr, Br, o, v, naux, opt)
    B.ccsd_destroy(h)


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_relaxed_couplings_match_oracle(precision):
    # strong two-electron integrals (kappa ~ 0.06), real well-separated roots, and an
    # orbital term of about 1 % of the coupling
    o, v, naux = 3, 8, 16
    H = make_hamiltonian(o, v, naux, seed=16, bscale=0.3)
    U, hr, Br, _ = B.ccsd_scf(H.eps, H.h, H.B, o, v, naux, tol=1e-13)
    h1, B1 = B.ccsd_rotate_integrals(U, H.h1, H.B1, o, v, naux)
    pairs = [(1, 2), (2, 1), (0, 1), (1, 0), (2, 0)]
    kw = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)
    if precision == B.PREC_MIXED:
        kw.update(splits=3, tc_min_flops=0.0, refine=1)
    F, Fu, KB = {}, {}, {}
    for relax in (1, 0):
        h = B.ccsd_create(H.eps, hr, Br, o, v, naux, B.ccsd_default_options(precision=precision, relax_orbitals=relax,
                                                                             **kw))
        try:
            B.ccsd_solve_ground(h)
            B.eom_solve_right(h, 2)
            B.eom_solve_left(h, 2)
            for kl in pairs:
                f = B.ccsd_derivative_coupling(h, kl[0], kl[1], 1, h1, B1)[0]
                if relax:
                    F[kl] = f
                    KB[kl] = B.ccsd_get_orbital_multipliers(h, kl[0], kl[1], o, v)
                else:
                    Fu[kl] = f
        finally:
            B.ccsd_destroy(h)
    # the oracle from its own Hartree-Fock orbitals (equal to the library's, first test)
    _, Uo, ho, Bo = rx.scf(H.h, H.B, o)
    h1o, B1o = rx.rotate(H.h1, H.B1, Uo)
    S = System(H.eps, ho, Bo, o)
    res = S.run(2, dense=True, tol=1e-12, tol_lin=1e-12)
    for kl in pairs:
        ref, kb = rx.relaxed_coupling(S, res, kl[0], kl[1], h1o, B1o, tol_lin=1e-12)
        assert abs(F[kl] - ref) < 1e-7 * abs(ref) + 1e-10, (kl, F[kl], ref)
        # kappa-bar is linear in the eigenvectors, so it carries their error to first
        # order: an absolute error up to about the eigenvector residual tolerance.  The
        # coupling is stationary in the multipliers and carries it only to second order.
        assert np.abs(KB[kl] - kb.numpy()).max() < 1e-7 * np.abs(kb.numpy()).max() + kw["tol_eom"]
        # the orbital term is resolved
        assert abs(F[kl] - Fu[kl]) > 100 * abs(F[kl] - ref)
