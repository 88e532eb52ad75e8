"""Pins of the oracle's learned-guess network (CPU only).

The gradient is pinned by central finite differences of the loss, the forward
pass by a network reduced to one hidden path (a closed form in scalar tanh),
the bf16 rounding by exactly representable halfway cases and by torch's own
conversion, and the features by the CCSD doubles residual at zero amplitudes,
which equals (ai|bj) (Eq. for Omega at T = 0: only the bare integral survives).
"""
import math

import numpy as np
import pytest
import torch

from oracle import mlp
from oracle import ccsd as occ
from paper_2301_13264_gb300.synth import make_hamiltonian


def _random_model(rng, wscale=0.4):
    m = np.zeros(mlp.N_PARAMS)
    m[:mlp.N_TRAIN] = rng.normal(0.0, wscale, mlp.N_TRAIN)
    m[mlp.N_TRAIN:mlp.N_TRAIN + 3] = rng.normal(0.0, 1.0, 3)        # mean
    m[mlp.N_TRAIN + 3:mlp.N_TRAIN + 6] = rng.uniform(0.5, 2.0, 3)   # scale
    m[mlp.N_TRAIN + 6] = 0.7                                        # target scale
    return m


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    m = _random_model(rng, 0.15)
    X = rng.normal(0.0, 1.5, (9, 3))
    T = rng.normal(0.0, 0.5, 9)
    _, g = mlp.loss_and_grad(m, X, T)
    # every first-layer weight and bias, the output layer, and a sample of W2
    probe = list(range(0, 3 * 128 + 128)) + list(range(mlp.N_TRAIN - 129, mlp.N_TRAIN))
    probe += list(rng.choice(np.arange(512, 512 + 128 * 128 + 128), 200, replace=False))
    h = 1e-6
    for k in probe:
        mp, mm = m.copy(), m.copy()
        mp[k] += h
        mm[k] -= h
        fd = (mlp.loss_and_grad(mp, X, T)[0] - mlp.loss_and_grad(mm, X, T)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-6 * abs(fd), (k, fd, g[k])


def test_loss_is_mean_squared_error_of_forward():
    rng = np.random.default_rng(4)
    m = _random_model(rng)
    X = rng.normal(0.0, 1.0, (11, 3))
    T = rng.normal(0.0, 1.0, 11)
    L, _ = mlp.loss_and_grad(m, X, T)
    y = mlp.forward(m, X)
    tscale = m[-1]
    assert L == pytest.approx(np.mean(((y - T) / tscale) ** 2), rel=1e-13)


def test_forward_single_path_closed_form():
    rng = np.random.default_rng(5)
    m = np.zeros(mlp.N_PARAMS)
    W1_0 = rng.normal(0, 1, 3)
    b1_0, w2_00, b2_0, w3_0, b3 = 0.3, -1.7, 0.2, 2.5, -0.4
    m[0:3] = W1_0
    m[384] = b1_0
    m[512] = w2_00                      # W2[0][0]
    m[512 + 128 * 128] = b2_0           # b2[0]
    m[512 + 128 * 128 + 128] = w3_0     # w3[0]
    m[mlp.N_TRAIN - 1] = b3
    mean = np.array([0.1, -0.2, 0.3])
    scale = np.array([2.0, 0.5, 1.0])
    m[mlp.N_TRAIN:mlp.N_TRAIN + 3] = mean
    m[mlp.N_TRAIN + 3:mlp.N_TRAIN + 6] = scale
    m[-1] = 3.0
    X = rng.normal(0, 1, (5, 3))
    y = mlp.forward(m, X)
    for r in range(5):
        xn = [(X[r, d] - mean[d]) / scale[d] for d in range(3)]
        a1 = math.tanh(sum(W1_0[d] * xn[d] for d in range(3)) + b1_0)
        expect = (w3_0 * math.tanh(w2_00 * a1 + b2_0) + b3) * 3.0
        assert y[r] == pytest.approx(expect, rel=1e-14)


def test_bf16_rounding():
    # halfway cases between neighbours 1, 1 + 2^-7, 1 + 2^-6 round to the even one
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -8 + 2 ** -20, 0.0],
                    dtype=np.float32)
    got = mlp.round_bf16(vals)
    assert list(got) == [1.0, 1.0, 1 + 2 ** -6, -1.0, 1 + 2 ** -7, 0.0]
    x = np.random.default_rng(6).normal(0, 3, 10000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.round_bf16(x), ref)


def test_features_from_zero_amplitude_residual():
    Hm = make_hamiltonian(3, 5, 11, seed=2)
    X = mlp.features(Hm)
    o, v = 3, 5
    t1 = torch.zeros(o, v, dtype=torch.float64)
    t2 = torch.zeros(o, o, v, v, dtype=torch.float64)
    _, om2, _ = occ.residual(t1, t2, torch.as_tensor(Hm.h), torch.as_tensor(Hm.B), o)
    g = om2.numpy()
    eps = Hm.eps
    for i in range(o):
        for j in range(o):
            for a in range(v):
                for b in range(v):
                    D = eps[o + a] + eps[o + b] - eps[i] - eps[j]
                    assert X[i, j, a, b, 1] == pytest.approx(D, rel=1e-14)
                    assert X[i, j, a, b, 0] == pytest.approx(-g[i, j, a, b] / D, rel=1e-10, abs=1e-14)
                    assert X[i, j, a, b, 2] == pytest.approx(abs(g[i, j, a, b]), rel=1e-10, abs=1e-14)


def test_inference_arithmetic_within_rounding_bound():
    # bf16 rounding of every first-layer activation (|h1| <= 1, error <= 2^-9 each)
    # moves a prediction by at most 2^-9 sum_jk |w3_j W2_jk| tscale
    rng = np.random.default_rng(8)
    m = _random_model(rng, 0.2)
    X = rng.normal(0.0, 1.0, (300, 3)).astype(np.float32)
    a = mlp.forward_inference(m, X)
    b = mlp.forward(mlp.bf16_weights(m), X)
    W1, b1, W2, b2, w3, b3, mean, scale, tscale = mlp.unpack(mlp.bf16_weights(m))
    bound = 2.0 ** -9 * float(np.sum(np.abs(w3)[:, None] * np.abs(W2))) * abs(tscale)
    assert np.abs(a - b).max() <= bound
    assert np.abs(a - b).max() > 0  # the rounding is really applied
