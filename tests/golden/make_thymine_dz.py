"""Write thymine_dz.json: the oracle's FP64 results at o=33, v=123, naux=550.

The thymine/cc-pVDZ-shaped synthetic Hamiltonian (seed 0, a 0.25 Eh gap between
the two lowest virtual orbitals) run through the whole oracle pipeline:

* ground state Omega(t) = 0 to max |Omega| < 1e-11 and E_CCSD (Theory section);
* Lambda, lambda^T A = -eta^T, to 1e-10 (left ground state, i = 0);
* the four lowest EOM-CCSD roots, right and left, Davidson to a residual norm of
  1e-9, biorthonormalised with the state conventions of the oracle (unit packed
  norm of R_k, largest component positive, L_k^T R_l = delta_kl,
  R_0^k = eta^T R_k / omega_k);
* the derivative coupling F_kl of Eq. NAC_NC along (h1, B1) for every ordered
  pair k != l of {0, 1, 2, 3, 4}, zeta solved to 1e-10.

Only the oracle and the seeded generator are imported.  The file is rewritten
after each coupling, so an interrupted run keeps the pairs already done; the
GPU test compares the pairs it finds.  Several hours on eight host cores.

    python tests/golden/make_thymine_dz.py [out.json]
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from oracle.solvers import System, Vec  # noqa: E402
from paper_2301_13264_gb300.synth import WORKLOADS, workload  # noqa: E402

NROOTS = 4
TOL_RES, TOL_EOM, TOL_LIN = 1e-11, 1e-9, 1e-10
# pairs in the order written: excited-excited first, then ground-excited and excited-ground
PAIRS = ([(k, l) for k in range(1, NROOTS + 1) for l in range(1, NROOTS + 1) if k != l]
         + [(0, l) for l in range(1, NROOTS + 1)] + [(k, 0) for k in range(1, NROOTS + 1)])


def singles_guesses(S: System, n: int):
    """Unit singles vectors on the n smallest orbital-energy differences."""
    order = torch.argsort(S.d1.reshape(-1))[:n]
    out = []
    for k in order:
        g = Vec.zeros(S.o, S.v)
        g.x1.view(-1)[k] = 1.0
        out.append(g)
    return out


def main(path: str) -> None:
    H = workload("thymine_dz")
    S = System(H.eps, H.h, H.B, H.o, vvvv_batch=16)
    out = {"workload": "thymine_dz", "params": WORKLOADS["thymine_dz"], "nroots": NROOTS,
           "tol": {"res": TOL_RES, "eom": TOL_EOM, "lin": TOL_LIN},
           "source": "oracle (tests/golden/make_thymine_dz.py)", "F": {}, "seconds": {}}

    def save():
        with open(path + ".tmp", "w") as f:
            json.dump(out, f, indent=1)
        os.replace(path + ".tmp", path)

    t0 = time.time()
    from oracle.solvers import Result
    res = Result()
    res.t, res.e_ccsd, res.iters["ground"] = S.solve_ground(tol=TOL_RES)
    res.lam, res.iters["lambda"] = S.solve_lambda(res.t, tol=TOL_LIN)
    out["e_ccsd"] = res.e_ccsd
    out["seconds"]["ground+lambda"] = time.time() - t0
    print(f"E = {res.e_ccsd!r}  ({time.time() - t0:.0f} s)", flush=True)
    save()
    # the four lowest roots, started from twice as many singles guesses so that none is missed
    t1 = time.time()
    omega_r, R, _ = S.davidson(lambda x: S.right(res.t, x), NROOTS, tol=TOL_EOM,
                               guesses=singles_guesses(S, 2 * NROOTS))
    omega_l, L, _ = S.davidson(lambda x: S.left(res.t, x), NROOTS, tol=TOL_EOM,
                               guesses=singles_guesses(S, 2 * NROOTS))
    res.omega, res.right, res.left = S.eom_from_vectors(res.t, omega_r, R, omega_l, L)
    out["omega"] = [float(w) for w in res.omega]
    out["omega_left"] = [float(w) for w in omega_l]
    out["r0"] = [float(s.c0) for s in res.right]
    out["seconds"]["eom"] = time.time() - t1
    print(f"omega = {out['omega']}  ({time.time() - t1:.0f} s)", flush=True)
    save()
    for (k, l) in PAIRS:
        t2 = time.time()
        F = S.coupling(res, k, l, H.h1, H.B1, tol_lin=TOL_LIN)
        out["F"][f"{k},{l}"] = float(F)
        out["seconds"][f"F{k},{l}"] = time.time() - t2
        print(f"F[{k},{l}] = {F!r}  ({time.time() - t2:.0f} s)", flush=True)
        save()
    out["seconds"]["total"] = time.time() - t0
    save()


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "thymine_dz.json"))
