"""The allocation-free coupling entry point against the regular one.

ccsd_derivative_coupling_noalloc serves callers that cannot allocate device
memory when they need a coupling (a dynamics loop inside another framework's
memory pool, or one that must not touch the allocator between steps).  It uses
a fixed scratch array in the library's device image instead of allocating.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2301_13264_gb300 import binding as B
from paper_2301_13264_gb300.synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def test_noalloc_coupling_matches_regular_entry_point_twice():
    assert torch.cuda.is_available()
    o, v, naux = 3, 7, 10
    H = make_hamiltonian(o, v, naux, seed=9)
    n = o + v
    rng = np.random.default_rng(4)
    extra = rng.normal(size=(n, n))
    dh = np.stack([H.h1, 0.5 * (extra + extra.T), np.zeros((n, n))])
    dB = np.stack([H.B1, np.zeros_like(H.B1), 0.3 * H.B1])
    dh_d = torch.as_tensor(dh, device="cuda")
    dB_d = torch.as_tensor(dB, device="cuda")
    opt = B.ccsd_default_options(tol_res=1e-11, tol_eom=1e-9, tol_lin=1e-11)
    h = B.ccsd_create(H.eps, H.h, H.B, o, v, naux, opt)
    try:
        B.ccsd_solve_ground(h)
        B.eom_solve_right(h, 2)
        B.eom_solve_left(h, 2)
        for (k, l) in [(1, 2), (0, 1)]:
            ref = B.ccsd_derivative_coupling(h, k, l, 3, dh_d, dB_d)
            B.ccsd_coupling_densities(h, k, l, np.zeros((n, n)))
            first = B.ccsd_derivative_coupling_noalloc(h, k, l, 3, dh_d, dB_d)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            B.ccsd_profile_start(h)
            second = B.ccsd_derivative_coupling_noalloc(h, k, l, 3, dh_d, dB_d)
            launched = B.ccsd_profile_stop(h)["launches"]
            # the second call changes nothing in the device's free memory
            assert torch.cuda.mem_get_info()[0] == free_before
            assert launched == 4 * 3 + 1
            for got in (first, second):
                for a, b in zip(got, ref):
                    assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
        # misuse is reported, not allocated around
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_derivative_coupling_noalloc(h, 2, 1, 1, dh_d, dB_d)
        assert e.value.status == B.ERR_STATE
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_derivative_coupling_noalloc(h, 0, 1, 1, dh, dB)
        assert e.value.status == B.ERR_ARG
        with pytest.raises(B.CCSDError) as e:
            B.ccsd_derivative_coupling_noalloc(h, 0, 1, 257, dh_d, dB_d)
        assert e.value.status == B.ERR_ARG
    finally:
        B.ccsd_destroy(h)
