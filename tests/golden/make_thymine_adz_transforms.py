"""Write thymine_adz_transforms.json: sampled oracle Jacobian transforms at o=33, v=228, naux=900.

The thymine/aug-cc-pVDZ-shaped synthetic Hamiltonian (seed 0) at seeded random
amplitudes t; one right transform A R and one left transform L^T A (Eq. for A)
of seeded random vectors R and L, each a full FP64 oracle evaluation.  The
vectors are too large to store (5.7e7 elements each), so the file keeps

* the elements at 4096 seeded random positions of the unpacked vector
  (singles [i][a] then doubles [i][j][a][b]) plus the 64 largest in magnitude;
* the largest magnitude, the packed norm and the plain sum over all elements,
  properties of the whole output.

Inputs: `random_amplitudes(33, 228, 22, scale=0.01, nvec=3)` gives t (vector 0),
R (vector 1) and L (vector 2).  Only the oracle and the seeded generator are
imported.  About ten minutes on eight host cores.

    python tests/golden/make_thymine_adz_transforms.py [out.json]
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from oracle import ccsd as cc  # noqa: E402
from oracle.solvers import System, Vec  # noqa: E402
from paper_2301_13264_gb300.synth import WORKLOADS, random_amplitudes, workload  # noqa: E402

SEED_VECTORS = 22
SEED_SAMPLE = 7
NSAMPLE, NTOP = 4096, 64


def summary(y: Vec, rng_seed: int):
    flat = torch.cat([y.x1.reshape(-1), y.x2.reshape(-1)]).numpy()
    rng = np.random.default_rng(rng_seed)
    idx = rng.choice(flat.size, NSAMPLE, replace=False)
    top = np.argsort(-np.abs(flat))[:NTOP]
    idx = np.unique(np.concatenate([idx, top]))
    return {"index": [int(i) for i in idx], "value": [float(flat[i]) for i in idx],
            "maxabs": float(np.abs(flat).max()), "packed_norm": y.norm(), "sum": float(flat.sum())}


def main(path: str) -> None:
    H = workload("thymine_adz")
    o, v = H.o, H.v
    S = System(H.eps, H.h, H.B, o, vvvv_batch=24)
    X1, X2 = random_amplitudes(o, v, SEED_VECTORS, scale=0.01, nvec=3)
    vec = [Vec(cc.as_t(X1[k]), cc.as_t(X2[k])) for k in range(3)]
    out = {"workload": "thymine_adz", "params": WORKLOADS["thymine_adz"],
           "inputs": f"random_amplitudes(o, v, {SEED_VECTORS}, scale=0.01, nvec=3): t = 0, R = 1, L = 2",
           "source": "oracle (tests/golden/make_thymine_adz_transforms.py)", "seconds": {}}
    t0 = time.time()
    out["right"] = summary(S.right(vec[0], vec[1]), SEED_SAMPLE)
    out["seconds"]["right"] = time.time() - t0
    print(f"right transform {time.time() - t0:.0f} s", flush=True)
    t0 = time.time()
    out["left"] = summary(S.left(vec[0], vec[2]), SEED_SAMPLE + 1)
    out["seconds"]["left"] = time.time() - t0
    print(f"left transform {time.time() - t0:.0f} s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                            "thymine_adz_transforms.json"))
