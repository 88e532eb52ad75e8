"""Learned starting doubles for the amplitude equations.

The ground-state solve normally starts from the first-order doubles
t_ij^ab = -(ia|jb)/D_ij^ab (D = e_a + e_b - e_i - e_j).  A small network,
trained on amplitudes the library itself converged, predicts per element the
correction t_CCSD - t_MP2 from the features (t_MP2, D, |(ia|jb)|); the solve then
starts from t_MP2 + correction.  The multiplier equations (Lambda, zeta) take the
same network on the features of their Jacobi start -rhs/D, trained on converged
ground multipliers.  Features, targets, starts, training and inference all run in
the library (``ccsd_guess_targets``, ``ccsd_guess_doubles``, ``ccsd_mlp_train``,
``ccsd_mlp_predict``); this module only gathers the training rows and moves arrays.  The converged amplitudes do not depend on the
start: the residual criterion of the solve is unchanged, and with no model set
the solve starts from the first-order guess.
"""
from __future__ import annotations

import numpy as np

from . import binding as _b
from .synth import Hamiltonian

__all__ = ["training_rows", "generate", "train", "guess_doubles", "save", "load"]


def training_rows(h, o: int, v: int, rows: int | None = None, rng: np.random.Generator | None = None,
                  which: int = _b.GUESS_AMPLITUDES):
    """(X[m, 3], T[m]) from a handle whose ground state has been solved.

    The library forms both: the features of the start and T = converged doubles - start
    doubles in [i][j][a][b] order (which = GUESS_AMPLITUDES: t2 from t_MP2;
    GUESS_MULTIPLIERS: lambda from -eta/D).  ``rows`` subsamples uniformly (without
    replacement) when given.
    """
    n2 = o * o * v * v
    X = np.zeros((n2, 3), dtype=np.float32)
    T = np.zeros(n2, dtype=np.float32)
    _b.ccsd_guess_targets(h, which, X, T)
    if rows is not None and rows < n2:
        rng = rng or np.random.default_rng(0)
        sel = np.sort(rng.choice(n2, rows, replace=False))
        X, T = X[sel], T[sel]
    return np.ascontiguousarray(X), np.ascontiguousarray(T)


def generate(hamiltonians, options=None, rows_per_system: int | None = None, seed: int = 0,
             which: int = _b.GUESS_AMPLITUDES):
    """Solve each Hamiltonian's ground state (and multipliers) and stack its training rows."""
    rng = np.random.default_rng(seed)
    xs, ts = [], []
    for Hm in hamiltonians:
        assert isinstance(Hm, Hamiltonian)
        h = _b.ccsd_create(Hm.eps, Hm.h, Hm.B, Hm.o, Hm.v, Hm.naux, options)
        try:
            _b.ccsd_solve_ground(h)
            X, T = training_rows(h, Hm.o, Hm.v, rows_per_system, rng, which)
        finally:
            _b.ccsd_destroy(h)
        xs.append(X)
        ts.append(T)
    return np.ascontiguousarray(np.concatenate(xs)), np.ascontiguousarray(np.concatenate(ts))


def train(X, T, steps: int = 3000, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Train on the GPU; returns (model float32[MLP_PARAMS], final mean squared error)."""
    return _b.ccsd_mlp_train(np.ascontiguousarray(X, dtype=np.float32), np.ascontiguousarray(T, dtype=np.float32),
                             steps, batch, lr, seed)


def guess_doubles(h, o: int, v: int, model=None, which: int = _b.GUESS_AMPLITUDES):
    """The starting doubles [o, o, v, v] the solve would use (the plain start without a model)."""
    x2 = np.zeros(o * o * v * v)
    _b.ccsd_guess_doubles(h, which, model, x2)
    return x2.reshape(o, o, v, v)


def save(model, path):
    np.save(path, np.asarray(model, dtype=np.float32))


def load(path):
    m = np.load(path).astype(np.float32)
    if m.shape != (_b.MLP_PARAMS,):
        raise ValueError(f"model file must hold {_b.MLP_PARAMS} floats")
    return m
