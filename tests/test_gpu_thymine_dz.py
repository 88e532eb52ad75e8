"""Full-size parity on the thymine/cc-pVDZ-shaped system (o=33, v=123, naux=550, a 0.25 Eh gap
between the two lowest virtual orbitals) against the oracle's stored FP64 results.

tests/golden/make_thymine_dz.py runs the oracle's whole pipeline (ground state to 1e-11,
Lambda and zeta to 1e-10, four EOM roots to a residual norm of 1e-9) and stores E_CCSD, the
four omega_k and the derivative couplings F_kl of Eq. NAC_NC along (h1, B1) for ordered pairs
of {0, 1, 2, 3, 4}, rewriting the file after each coupling; these tests compare what the file
holds.  The GPU forms must match within the method's FP64 tolerances: 1e-8 Eh on the energy,
1e-8 on excitation energies and 1e-7 relative on couplings.
"""
import json
import os

import numpy as np
import pytest

from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "thymine_dz.json")
# The roots are converged ten times below the stored ones' 1e-9: a root refined on its own keeps a
# component along a neighbouring root of about |r| / (omega_l - omega_k), which a coupling of the
# two carries at first order, while the oracle's Rayleigh-Ritz step over all four roots removes it.
TOL = dict(tol_res=1e-10, tol_eom=1e-10, tol_lin=1e-10, max_iter=200, davidson_max_sub=96)
TOL_PAIRS = dict(TOL, tol_eom=1e-9)  # the eigenpair check below needs the residual only


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def run_form(golden, pairs, **opt):
    """E, the stored roots (when the file holds them) and the couplings of `pairs` in one handle.

    One root more than stored is solved and each stored root is matched to the nearest solved
    one, so that a root the two Davidson solvers order or find differently above the stored
    ones does not decide the comparison; the stored root indices are mapped to the library's."""
    H = workload("thymine_dz")
    h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**TOL, **opt))
    try:
        e, _ = B.ccsd_solve_ground(h)
        w, F = None, {}
        if "omega" in golden:
            n = golden["nroots"] + 1
            wg, _ = B.eom_solve_right(h, n)
            B.eom_solve_left(h, n)
            idx = [int(np.argmin(np.abs(np.array(wg) - x))) for x in golden["omega"]]
            assert len(set(idx)) == len(idx), (wg, golden["omega"])
            w = [wg[i] for i in idx]
            m = [0] + [i + 1 for i in idx]  # stored state index -> library state index
            F = {kl: B.ccsd_derivative_coupling(h, m[kl[0]], m[kl[1]], 1, H.h1, H.B1)[0] for kl in pairs}
    finally:
        B.ccsd_destroy(h)
    return e, w, F


def check(golden, e, w, F):
    assert abs(e - golden["e_ccsd"]) < 1e-8, (e, golden["e_ccsd"])
    if w is not None:
        assert np.abs(np.array(w) - np.array(golden["omega"])).max() < 1e-8, (w, golden["omega"])
    for kl, f in F.items():
        ref = golden["F"][f"{kl[0]},{kl[1]}"]
        assert abs(f - ref) < 1e-7 * abs(ref), (kl, f, ref)


def stored_pairs(golden, limit=None):
    pairs = [tuple(int(x) for x in k.split(",")) for k in golden["F"]]
    return pairs[:limit] if limit else pairs


def test_thymine_dz_refined_mixed_matches_oracle(golden):
    """Split-bf16 tensor-core products with FP64 refinement of every solve: the energy, the four
    roots and every stored coupling."""
    e, w, F = run_form(golden, stored_pairs(golden), precision=B.PREC_MIXED, splits=3)
    check(golden, e, w, F)


def test_thymine_dz_fp64_grade_matches_oracle(golden):
    """Every contraction as FP64-grade tensor-core products, solved directly to the FP64
    tolerances: the energy, the four roots and up to four stored couplings."""
    e, w, F = run_form(golden, stored_pairs(golden, 4), precision=B.PREC_FP64_TC)
    check(golden, e, w, F)


def test_thymine_dz_fp64_ground_state_matches_oracle(golden):
    """The plain FP64 (DFMA) form's ground-state energy (its EOM roots at this size take minutes
    each; the FP64-grade form above covers them)."""
    H = workload("thymine_dz")
    h = B.ccsd_create(H.eps, H.h, H.B, H.o, H.v, H.naux, B.ccsd_default_options(**TOL))
    try:
        e, _ = B.ccsd_solve_ground(h)
    finally:
        B.ccsd_destroy(h)
    assert abs(e - golden["e_ccsd"]) < 1e-8


def test_thymine_dz_eigenpairs_against_the_oracle_jacobian():
    """The refined mixed form's two lowest roots, checked with the oracle's own Jacobian at the
    library's converged amplitudes: |A R_k - omega_k R_k| and |L_k^T A - omega_k L_k^T| are at
    the EOM threshold (1e-9) relative to the vectors (bound 1e-8 for the plain 2-norm against
    the solver's metric)."""
    from oracle import ccsd as cc
    from oracle.solvers import System, Vec

    H = workload("thymine_dz")
    o, v = H.o, H.v
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux,
                      B.ccsd_default_options(**TOL_PAIRS, precision=B.PREC_MIXED, splits=3))
    try:
        B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        wl, _ = B.eom_solve_left(h, 2)
        dim = o * v + o * o * v * v
        t = np.zeros(dim)
        B.ccsd_get_amplitudes(h, t)
        R, L = np.zeros((2, dim)), np.zeros((2, dim))
        B.ccsd_get_states(h, 2, R, L)
    finally:
        B.ccsd_destroy(h)
    S = System(H.eps, H.h, H.B, o, vvvv_batch=16)

    def vec(x):
        return Vec(cc.as_t(x[:o * v].reshape(o, v)), cc.as_t(x[o * v:].reshape(o, o, v, v)))

    def flat(x):
        return np.concatenate([x.x1.numpy().reshape(-1), x.x2.numpy().reshape(-1)])

    tv = vec(t)
    for k in range(2):
        ar = flat(S.right(tv, vec(R[k])))
        la = flat(S.left(tv, vec(L[k])))
        assert np.linalg.norm(ar - w[k] * R[k]) < 1e-8 * np.linalg.norm(R[k]), k
        assert np.linalg.norm(la - wl[k] * L[k]) < 1e-8 * np.linalg.norm(L[k]), k
    assert abs(w[0] - wl[0]) < 1e-9 and abs(w[1] - wl[1]) < 1e-9
