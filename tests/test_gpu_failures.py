"""Failure statuses of the library, each caused on the host, and the allocator callbacks.

* CCSD_ERR_OOM: allocator callbacks (ccsd_options.alloc / free / alloc_ctx) that refuse
  above a cap; the same handle works again once the cap is lifted, and every block the
  library took is returned by ccsd_destroy.
* CCSD_ERR_DEGENERATE: tol_degen above the gap between the two roots, whose difference
  the coupling multiplier gamma = L_i / (omega_j - omega_i) divides by.
* CCSD_ERR_TIMEOUT: a short wait budget and a GEMM whose producer withholds its operand
  loads (ccsd_inject_stall): the MMA issuer's bounded wait runs out, the kernel raises
  its flag and exits, and the call reports it; with the default budget the same handle
  then gives the oracle's transform.  No fault, trap or hang is involved.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd as cc
from oracle.solvers import System, Vec
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    assert torch.cuda.is_available()
    B.lib()


class CappedAllocator:
    """Device memory from torch's caching allocator on the handle's stream, refused once the
    live total would exceed `cap` bytes; counts every block."""

    def __init__(self, cap=None):
        self.cap = cap
        self.live = {}
        self.calls = 0
        self.refused = 0
        self.alloc_fn = B.ALLOC_FN(self._alloc)
        self.free_fn = B.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.cap is not None and sum(self.live.values()) + nbytes > self.cap:
            self.refused += 1
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        self.live[p] = int(nbytes)
        return p

    def _free(self, p, stream, ctx):
        nbytes = self.live.pop(p)
        assert nbytes > 0
        torch.cuda.caching_allocator_delete(p)

    def options(self, **kw):
        return B.ccsd_default_options(alloc=self.alloc_fn, free=self.free_fn, **kw)


TIGHT = dict(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11, max_iter=200)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_allocator_callbacks_carry_every_block_and_oom(precision):
    H = make_hamiltonian(3, 7, 10, seed=12)
    extra = dict(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0) if precision == "mixed" else {}
    ref = B.ccsd_create(H.eps, H.h, H.B, 3, 7, 10, B.ccsd_default_options(**TIGHT, **extra))
    try:
        e_ref, _ = B.ccsd_solve_ground(ref)
        w_ref, _ = B.eom_solve_right(ref, 2)
        B.eom_solve_left(ref, 2)
        F_ref = B.ccsd_derivative_coupling(ref, 1, 2, 1, H.h1, H.B1)[0]
    finally:
        B.ccsd_destroy(ref)
    A = CappedAllocator()
    h = B.ccsd_create(H.eps, H.h, H.B, 3, 7, 10, A.options(**TIGHT, **extra))
    try:
        created = sum(A.live.values())
        assert A.calls > 0 and created > 0
        # below what the ground-state solve needs: refused, reported as out of memory
        A.cap = created + 1024
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_solve_ground(h)
        assert err.value.status == B.ERR_OOM and A.refused > 0
        # the handle is still usable once memory is available again
        A.cap = None
        e, _ = B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        F = B.ccsd_derivative_coupling(h, 1, 2, 1, H.h1, H.B1)[0]
    finally:
        B.ccsd_destroy(h)
    torch.cuda.synchronize()
    assert A.live == {}, f"{len(A.live)} blocks not returned by ccsd_destroy"
    assert abs(e - e_ref) < 1e-10
    assert np.abs(np.array(w) - np.array(w_ref)).max() < 1e-9
    assert abs(F - F_ref) < 1e-8 * abs(F_ref)


def test_allocator_needs_both_callbacks():
    H = make_hamiltonian(2, 4, 6, seed=1)
    A = CappedAllocator()
    with pytest.raises(B.CCSDError) as err:
        B.ccsd_create(H.eps, H.h, H.B, 2, 4, 6, B.ccsd_default_options(alloc=A.alloc_fn))
    assert err.value.status == B.ERR_ARG
    h = B.ccsd_create(H.eps, H.h, H.B, 2, 4, 6, A.options())
    try:
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_batch_create([h], 2)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)


def test_degenerate_roots_are_reported():
    """gamma divides by omega_j - omega_i: with tol_degen above that gap the coupling of the
    two excited states is refused, while pairs with the ground state (gap omega) still work."""
    H = make_hamiltonian(3, 7, 10, seed=12)
    h = B.ccsd_create(H.eps, H.h, H.B, 3, 7, 10, B.ccsd_default_options(**TIGHT))
    try:
        B.ccsd_solve_ground(h)
        w, _ = B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
    finally:
        B.ccsd_destroy(h)
    gap = abs(w[1] - w[0])
    assert 0 < gap < min(w)
    h = B.ccsd_create(H.eps, H.h, H.B, 3, 7, 10, B.ccsd_default_options(**TIGHT, tol_degen=2.0 * gap))
    try:
        B.ccsd_solve_ground(h)
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_derivative_coupling(h, 1, 2, 1, H.h1, H.B1)
        assert err.value.status == B.ERR_DEGENERATE
        B.ccsd_derivative_coupling(h, 0, 1, 1, H.h1, H.B1)
    finally:
        B.ccsd_destroy(h)


def test_wait_budget_timeout_then_recovery():
    o, v, naux = 3, 9, 12
    H = make_hamiltonian(o, v, naux, seed=13)
    X1, X2 = random_amplitudes(o, v, 14, scale=0.03, nvec=2)
    t = np.concatenate([X1[0].ravel(), X2[0].ravel()])
    X = np.concatenate([X1[1].ravel(), X2[1].ravel()])[None]
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux,
                      B.ccsd_default_options(precision=B.PREC_MIXED, splits=3, tc_min_flops=0.0))
    try:
        B.ccsd_set_amplitudes(h, t, np.zeros_like(t))
        Y = np.zeros_like(X)
        # a short budget alone does not disturb a normal run
        B.ccsd_set_wait_budget(h, 20_000_000)
        B.ccsd_jacobian_transform(h, 0, 1, X, Y)
        Y_short = Y.copy()
        # a GEMM that never receives its operands: the bounded wait runs out (about 1 ms)
        B.ccsd_set_wait_budget(h, 2_000_000)
        B.ccsd_inject_stall(h)
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_jacobian_transform(h, 0, 1, X, np.zeros_like(X))
        assert err.value.status == B.ERR_TIMEOUT
        # default budget: the same handle works again
        B.ccsd_set_wait_budget(h, 0)
        Y = np.zeros_like(X)
        B.ccsd_jacobian_transform(h, 0, 1, X, Y)
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_set_wait_budget(h, -1)
        assert err.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
    S = System(H.eps, H.h, H.B, o)
    ar = S.right(Vec(cc.as_t(X1[0]), cc.as_t(X2[0])), Vec(cc.as_t(X1[1]), cc.as_t(X2[1])))
    ref = np.concatenate([ar.x1.numpy().ravel(), ar.x2.numpy().ravel()])
    for got in (Y_short[0], Y[0]):
        assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()
    h64 = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, B.ccsd_default_options())
    try:
        with pytest.raises(B.CCSDError) as err:
            B.ccsd_inject_stall(h64)
        assert err.value.status == B.ERR_STATE
    finally:
        B.ccsd_destroy(h64)


def test_complex_root_is_reported():
    """A strongly correlated system (o=2, v=8, integrals ten times the usual scale) whose two
    lowest EOM-CCSD roots are a complex-conjugate pair (the non-symmetric Jacobian's dense
    eigenvalues, from the oracle): the Davidson solve reports CCSD_ERR_COMPLEX_ROOT instead of
    returning real parts."""
    H = make_hamiltonian(2, 8, 20, seed=0, bscale=1.0, hnoise=0.2)
    S = System(H.eps, H.h, H.B, 2)
    t, _, _ = S.solve_ground(tol=1e-12, maxit=300)
    w = np.linalg.eigvals(S.dense_jacobian(t).numpy())
    low = w[np.argsort(w.real)[:2]]
    assert np.abs(low.imag).min() > 1e-2 and abs(low[0] - np.conj(low[1])) < 1e-10
    h = B.ccsd_create(H.eps, H.h, H.B, 2, 8, 20, B.ccsd_default_options(tol_res=1e-11, tol_eom=1e-8, max_iter=300))
    try:
        B.ccsd_solve_ground(h)
        with pytest.raises(B.CCSDError) as err:
            B.eom_solve_right(h, 2)
        assert err.value.status == B.ERR_COMPLEX_ROOT
    finally:
        B.ccsd_destroy(h)
