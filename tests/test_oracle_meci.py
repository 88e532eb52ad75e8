"""Crossing-point search (the application of the couplings in the paper's Results section) in the oracle.

Two electrons, where CC is exact: the Bearpark-Robb-Schlegel direction built from the CC oracle's
Lagrangian gradients and biorthonormal coupling equals the one built from full CI (Hellmann-Feynman
gradients and coupling), and the search driven by the FCI quantities ends at a point that satisfies the
crossing conditions checked with FCI energies alone: E_2 = E_1, and E_2 stationary along the seam tangent
(the direction orthogonal to g and h), by central differences.
"""
import numpy as np
import pytest

from oracle.fockspace import CCBruteForce
from oracle.meci import Family, bearpark_direction, cc_point, fci_point, search
from paper_2301_13264_gb300.synth import make_hamiltonian


@pytest.fixture(scope="module")
def family():
    # LUMO shift, LUMO/LUMO+1 coupling, and a random direction confined by a quadratic raise of
    # every virtual level, so that the crossing seam has a lowest point
    o, v, naux = 1, 4, 6
    H = make_hamiltonian(o, v, naux, seed=2)
    n = o + v
    Ea = np.zeros((n, n))
    Ea[1, 1] = 1.0
    Eb = np.zeros((n, n))
    Eb[1, 2] = Eb[2, 1] = 1.0
    rng = np.random.default_rng(3)
    Ec = rng.normal(0, 0.1, (n, n))
    Ec = (Ec + Ec.T) / 2
    Bc = rng.normal(0, 0.02, H.B.shape)
    Bc = (Bc + Bc.transpose(0, 2, 1)) / 2
    zero = np.zeros_like(H.B)
    return Family(H.eps, H.h, H.B, [(Ea, zero), (Eb, zero), (Ec, Bc)], o,
                  quad=[(0 * Ea, zero), (0 * Ea, zero), (np.diag([0.0] + [1.0] * v), zero)])


@pytest.fixture(scope="module")
def crossing(family):
    x, it, q = search(lambda x: fci_point(family, x), [0.5, 0.0, 0.0], step=0.3, tol=1e-9, maxit=500)
    return x, q


def _fci_energies(family, x):
    h, B = family.hamiltonian(x)
    return CCBruteForce(h, B, family.o).fci()[0]


def test_fci_search_meets_crossing_conditions(family, crossing):
    x, (E1, E2, g1, g2, f12) = crossing
    assert abs(E2 - E1) < 1e-9
    # seam tangent: orthogonal to g = grad(E2 - E1) and h = (E2 - E1) F_12 (h's direction is F_12's)
    g = g2 - g1
    t = np.cross(g, f12)
    t /= np.linalg.norm(t)
    d = 1e-3
    dE = (_fci_energies(family, x + d * t)[2] - _fci_energies(family, x - d * t)[2]) / (2 * d)
    assert abs(dE) < 1e-5
    # away from the seam the same difference is of order |grad E2|
    dEg = (_fci_energies(family, x + d * g / np.linalg.norm(g))[2] - E2) / d
    assert abs(dEg) > 1e-2


@pytest.mark.parametrize("x", [(0.5, 0.0, 0.1), (0.7, -0.05, -0.3)])
def test_cc_quantities_equal_fci_for_two_electrons(family, x):
    x = np.array(x)
    c, f = cc_point(family, x), fci_point(family, x)
    assert abs(c[0] - f[0]) < 1e-10 and abs(c[1] - f[1]) < 1e-10
    assert np.abs(c[2] - f[2]).max() < 1e-9 and np.abs(c[3] - f[3]).max() < 1e-9
    # the biorthonormal coupling is the FCI one times a state-scale factor: same direction
    cos = c[4] @ f[4] / (np.linalg.norm(c[4]) * np.linalg.norm(f[4]))
    assert abs(abs(cos) - 1.0) < 1e-12
    assert np.abs(bearpark_direction(*c) - bearpark_direction(*f)).max() < 1e-9


def test_cc_direction_and_h_vector_near_the_crossing(family, crossing):
    """Approaching the crossing along g: the CC direction follows the FCI one and vanishes linearly,
    and h = (E_2 - E_1) F_12 stays finite while F_12 itself grows as 1/(E_2 - E_1)."""
    x, (E1, E2, g1, g2, f12) = crossing
    q = (g2 - g1) / np.linalg.norm(g2 - g1)
    hn, fn = [], []
    for d in (1e-2, 1e-3):
        c, f = cc_point(family, x + d * q), fci_point(family, x + d * q)
        G = bearpark_direction(*c)
        assert np.abs(G - bearpark_direction(*f)).max() < 1e-8
        assert np.linalg.norm(G) < 2.5 * np.linalg.norm(g2 - g1) * d  # the gap term, 2 |g| d
        hn.append(np.linalg.norm((c[1] - c[0]) * c[4]))
        fn.append(np.linalg.norm(c[4]))
    assert abs(hn[1] / hn[0] - 1.0) < 0.05
    assert fn[1] > 5.0 * fn[0]
