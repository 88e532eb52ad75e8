"""Learned doubles guess: features, network and gradients (oracle, FP64 CPU).

Test infrastructure of the oracle; see the package docstring.

The learned start replaces the first-order (MP2-type) doubles guess
t_ij^ab = -(ia|jb) / D_ij^ab, D_ij^ab = e_a + e_b - e_i - e_j, by that guess plus
a correction predicted per element by a small network from three features:

    x_ijab = (t_MP2_ijab, D_ijab, |(ia|jb)|)

The network is 3 -> 128 -> 128 -> 1 with tanh hidden layers,

    xn = (x - mean) / scale
    h1 = tanh(W1 xn + b1),  h2 = tanh(W2 h1 + b2),  y = w3 . h2 + b3
    prediction = y * tscale,

and is trained on the mean squared error of y against target / tscale.  A model
is one flat float array: W1[128][3], b1[128], W2[128][128], b2[128], w3[128], b3,
mean[3], scale[3], tscale.  The first 17153 entries are trainable.

Nothing here is in the paper: the starting point of the amplitude iterations does
not change the solution the CCSD equations define, so the converged residual is
the criterion the learned start is evaluated by.
"""
from __future__ import annotations

import numpy as np

H = 128
N_PARAMS = H * 3 + H + H * H + H + H + 1 + 7
N_TRAIN = N_PARAMS - 7
_OW1, _OB1 = 0, H * 3
_OW2 = _OB1 + H
_OB2 = _OW2 + H * H
_OW3 = _OB2 + H
_OB3 = _OW3 + H


def unpack(model):
    """Views of the weights in FP64: (W1[128,3], b1, W2[128,128], b2, w3, b3, mean, scale, tscale)."""
    m = np.asarray(model, dtype=np.float64)
    if m.shape != (N_PARAMS,):
        raise ValueError(f"model must have {N_PARAMS} entries")
    return (m[_OW1:_OB1].reshape(H, 3), m[_OB1:_OW2], m[_OW2:_OB2].reshape(H, H), m[_OB2:_OW3],
            m[_OW3:_OB3], m[_OB3], m[N_TRAIN:N_TRAIN + 3], m[N_TRAIN + 3:N_TRAIN + 6], m[N_TRAIN + 6])


def round_bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the upper 16 bits of the IEEE binary32 pattern; rounding to
    nearest-even adds 0x7FFF plus the lowest kept bit before truncating.  Inputs
    are finite.
    """
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weights(model):
    """The model with its trainable weights rounded to bf16 (what inference uses)."""
    m = np.asarray(model, dtype=np.float32).astype(np.float64)
    m[:N_TRAIN] = round_bf16(np.asarray(model, dtype=np.float32)[:N_TRAIN])
    return m


def forward(model, X):
    """Predictions (target units) for features X[n, 3], FP64 arithmetic."""
    W1, b1, W2, b2, w3, b3, mean, scale, tscale = unpack(model)
    xn = (np.asarray(X, dtype=np.float64) - mean) / scale
    h1 = np.tanh(xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return (h2 @ w3 + b3) * tscale


def forward_inference(model, X):
    """Predictions of the inference arithmetic: every weight rounded to bf16, the first
    hidden layer's output rounded to bf16 (it is the operand of the second layer's
    bf16 product), everything else in FP64."""
    W1, b1, W2, b2, w3, b3, mean, scale, tscale = unpack(bf16_weights(model))
    xn = (np.asarray(X, dtype=np.float32).astype(np.float64) - mean) / scale
    h1 = round_bf16(np.tanh(xn @ W1.T + b1).astype(np.float32))
    h2 = np.tanh(h1 @ W2.T + b2)
    return (h2 @ w3 + b3) * tscale


def inference_flip_bound(model):
    """Largest change of one prediction when a single first-layer activation moves by
    one bf16 unit in the last place (2^-8 relative, |h1| <= 1): the inference kernel
    and forward_inference may round an activation that sits within FP32 rounding of
    a bf16 tie differently."""
    W1, b1, W2, b2, w3, b3, mean, scale, tscale = unpack(bf16_weights(model))
    return 2.0 ** -8 * float(np.max(np.sum(np.abs(w3)[:, None] * np.abs(W2), axis=0))) * abs(tscale)


def loss_and_grad(model, X, T):
    """(L, dL/dw[N_TRAIN]) for L = mean_r (y_r - T_r / tscale)^2, by reverse-mode chain rule."""
    W1, b1, W2, b2, w3, b3, mean, scale, tscale = unpack(model)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    xn = (X - mean) / scale
    h1 = np.tanh(xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ w3 + b3
    diff = y - T / tscale
    L = float(np.mean(diff * diff))
    dy = 2.0 * diff / n                       # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)  # dL/d(W2 h1 + b2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)        # dL/d(W1 xn + b1)
    g_W1 = dz1.T @ xn
    g_b1 = dz1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g


def features(H_):
    """X[o, o, v, v, 3] = (-(ia|jb)/D, D, |(ia|jb)|) for a Hamiltonian (eps, B, o).

    (ia|jb) = sum_P B^P_ia B^P_jb over the bare Cholesky factors; D from the
    orbital energies eps.  Element order [i][j][a][b].
    """
    o = H_.o
    eps = np.asarray(H_.eps, dtype=np.float64)
    Bov = np.asarray(H_.B, dtype=np.float64)[:, :o, o:]
    g = np.einsum("Pia,Pjb->ijab", Bov, Bov)
    D = eps[o:][None, None, :, None] + eps[o:][None, None, None, :] - eps[:o][:, None, None, None] \
        - eps[:o][None, :, None, None]
    return np.stack([-g / D, D, np.abs(g)], axis=-1)
