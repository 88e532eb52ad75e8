"""Batches of systems: one graph launch for the block transforms of every system.

The batched transforms replay the very kernels the single-system path launches,
so their results must equal that path's; the single-system path is itself
compared with the oracle in the parity tests, and one system here is checked
against the oracle directly.  The lockstep batched Davidson must find the same
roots and leave every handle ready for couplings, like the per-system solvers.
"""
import numpy as np
import pytest

from oracle import ccsd as cc
from oracle.solvers import System, Vec
from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian, random_amplitudes

pytestmark = pytest.mark.gpu

# uneven occupied / virtual counts, naux = 3.5 (o + v)
SHAPES = [(2, 9), (3, 14), (4, 11), (5, 20)]


def _flat(x1, x2):
    return np.concatenate([np.ravel(x1), np.ravel(x2)])


def _systems(precision, seed0=40, **kw):
    hs, Hs = [], []
    for k, (o, v) in enumerate(SHAPES):
        H = make_hamiltonian(o, v, int(3.5 * (o + v)), seed=seed0 + k)
        opt = B.ccsd_default_options(precision=precision, **kw)
        hs.append(B.ccsd_create(H.eps, H.h, H.B, o, v, H.naux, opt))
        Hs.append(H)
    return hs, Hs


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_batch_transform_matches_single_system_path(precision):
    nvec = 4
    kw = dict(tc_min_flops=0.0, autotune=1) if precision == B.PREC_MIXED else {}
    hs, Hs = _systems(precision, **kw)
    b = None
    try:
        t_all, xs = [], []
        for k, (h, H) in enumerate(zip(hs, Hs)):
            x1, x2 = random_amplitudes(H.o, H.v, 100 + k, scale=0.05, nvec=nvec + 1)
            t = _flat(x1[0], x2[0])
            B.ccsd_set_amplitudes(h, t, np.zeros_like(t))
            t_all.append((x1[0], x2[0]))
            xs.append(np.stack([_flat(x1[q + 1], x2[q + 1]) for q in range(nvec)]))
        ref = {}
        for side in (0, 1):
            ref[side] = []
            for h, x in zip(hs, xs):
                y = np.zeros_like(x)
                B.ccsd_jacobian_transform(h, side, nvec, x, y)
                ref[side].append(y)
        b = B.ccsd_batch_create(hs, nvec)
        for rep in range(3):  # first call runs directly and captures, later calls replay the graph
            for side in (0, 1):
                ys = [np.zeros_like(x) for x in xs]
                B.ccsd_batch_transform(b, side, xs, ys)
                for y, r in zip(ys, ref[side]):
                    assert _relerr(y, r) < 1e-13
        st = B.ccsd_batch_stats(b)
        assert st["captures"] == 2 and st["launches"] == 4 and st["nodes"] > len(hs)
    finally:
        B.ccsd_batch_destroy(b)
        for h in hs:
            B.ccsd_destroy(h)
    if precision == B.PREC_FP64:
        # the batched result of one system against the oracle
        H = Hs[1]
        S_ = System(H.eps, H.h, H.B, H.o)
        tv = Vec(cc.as_t(t_all[1][0]), cc.as_t(t_all[1][1]))
        x = xs[1][0]
        n1 = H.o * H.v
        r = Vec(cc.as_t(x[:n1].reshape(H.o, H.v)), cc.as_t(x[n1:].reshape(H.o, H.o, H.v, H.v)))
        ar = S_.right(tv, r)
        assert _relerr(ref[0][1][0], _flat(ar.x1.numpy(), ar.x2.numpy())) < 1e-12


def test_batch_eom_matches_per_system_solvers():
    nroots = 3
    hs, Hs = _systems(B.PREC_FP64, seed0=60, tol_eom=1e-8)
    hs2, _ = _systems(B.PREC_FP64, seed0=60, tol_eom=1e-8)
    b = None
    try:
        for h, h2 in zip(hs, hs2):
            B.ccsd_solve_ground(h)
            B.ccsd_solve_ground(h2)
        b = B.ccsd_batch_create(hs, 8)
        wr, itr = B.ccsd_batch_eom_solve(b, 0, nroots, len(hs))
        wl, itl = B.ccsd_batch_eom_solve(b, 1, nroots, len(hs))
        assert np.abs(wr - wl).max() < 1e-7
        assert min(itr) >= 1 and min(itl) >= 1
        st = B.ccsd_batch_stats(b)
        assert st["launches"] >= max(itr)  # at least one graph launch per iteration after the first
        for k, (h, h2, H) in enumerate(zip(hs, hs2, Hs)):
            w_ref, _ = B.eom_solve_right(h2, nroots)
            B.eom_solve_left(h2, nroots)
            assert np.abs(wr[k] - np.array(w_ref)).max() < 1e-8
            # couplings from the batch-solved handle equal the per-system ones
            for (p, q) in [(1, 2), (0, 1)]:
                f = B.ccsd_derivative_coupling(h, p, q, 1, H.h1, H.B1)[0]
                f2 = B.ccsd_derivative_coupling(h2, p, q, 1, H.h1, H.B1)[0]
                assert abs(f - f2) <= 1e-6 * abs(f2) + 1e-12
    finally:
        B.ccsd_batch_destroy(b)
        for h in hs + hs2:
            B.ccsd_destroy(h)


def test_batch_errors():
    hs, _ = _systems(B.PREC_FP64)
    try:
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_batch_create(hs, 17)
        assert e.value.status == B.ERR_ARG
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_batch_create([hs[0], hs[0]], 4)
        assert e.value.status == B.ERR_ARG
        b = B.ccsd_batch_create(hs, 2)
        try:
            xs = [np.zeros((2, B.vector_dim(o, v))) for o, v in SHAPES]
            with pytest.raises(B.CCSDError) as e:
                B.ccsd_batch_transform(b, 0, xs, [x.copy() for x in xs])
            assert e.value.status == B.ERR_STATE
            with pytest.raises(B.CCSDError) as e:
                B.ccsd_batch_eom_solve(b, 0, 3, len(hs))  # more roots than trial vectors per launch
            assert e.value.status == B.ERR_ARG
            with pytest.raises(B.CCSDError) as e:
                B.ccsd_batch_eom_solve(b, 0, 2, len(hs))  # no ground state yet
            assert e.value.status == B.ERR_STATE
        finally:
            B.ccsd_batch_destroy(b)
    finally:
        for h in hs:
            B.ccsd_destroy(h)
