"""Learned doubles guess on the GPU: kernels against the oracle, and what the guess gains.

The training gradient (FP32 kernels) is compared with the oracle's FP64
reverse-mode gradient, the inference kernel (bf16-rounded weights, FP32
accumulation) with the oracle's forward pass on the same rounded weights, and the
feature kernel with the oracle's features.  The last test trains a network on
amplitudes the library converged for several systems of one generator and checks,
on a held-out system of the same generator, that the learned start lies closer to
the converged amplitudes than the first-order start and that the solve from it
converges to the same amplitudes and energy under the same residual criterion.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2301_13264_gb300 import binding as b
from paper_2301_13264_gb300 import learned_guess as lg
from paper_2301_13264_gb300.synth import make_hamiltonian

pytestmark = pytest.mark.gpu


def _model(seed, wscale=0.3):
    rng = np.random.default_rng(seed)
    m = np.zeros(b.MLP_PARAMS, dtype=np.float32)
    m[:b.MLP_TRAINABLE] = rng.normal(0.0, wscale, b.MLP_TRAINABLE)
    m[b.MLP_TRAINABLE:b.MLP_TRAINABLE + 3] = rng.normal(0.0, 1.0, 3)
    m[b.MLP_TRAINABLE + 3:b.MLP_TRAINABLE + 6] = rng.uniform(0.5, 2.0, 3)
    m[b.MLP_TRAINABLE + 6] = 0.8
    return m


@pytest.mark.parametrize("n", [1, 7, 1003, 40000])
def test_gradient_matches_oracle(n):
    rng = np.random.default_rng(n)
    m = _model(11, 0.1)
    X = rng.normal(0.0, 1.5, (n, 3)).astype(np.float32)
    T = rng.normal(0.0, 0.6, n).astype(np.float32)
    loss, g = b.ccsd_mlp_gradient(m, X, T)
    L_ref, g_ref = omlp.loss_and_grad(m.astype(np.float64), X, T)
    assert loss == pytest.approx(L_ref, rel=1e-5)
    scale = np.abs(g_ref).max()
    err = np.abs(g.astype(np.float64) - g_ref)
    # FP32 products and sums over n rows and 128 hidden units: a few 1e-6 of the scale
    assert err.max() <= 1e-4 * scale, (err.max(), scale)


@pytest.mark.parametrize("n", [1, 5, 1003, 100001])
def test_predict_matches_oracle_with_bf16_weights(n):
    rng = np.random.default_rng(100 + n)
    m = _model(12)
    X = rng.normal(0.0, 1.5, (n, 3)).astype(np.float32)
    out = np.zeros(n, dtype=np.float32)
    b.ccsd_mlp_predict(m, X, out)
    ref = omlp.forward_inference(m, X)
    # bf16 weights and bf16 first-layer activations on both sides; FP32 accumulation in
    # the kernel and tanh from the hardware exponential and reciprocal (absolute error
    # below 1e-6).  An activation within that error of a bf16 tie may round the other
    # way: allow a few such flips per row, plus the tanh error through w3 and FP32 noise.
    err = np.abs(out - ref)
    w3 = np.abs(omlp.bf16_weights(m)[512 + 128 * 128 + 128:512 + 128 * 128 + 256]).sum()
    noise = 1e-6 * w3 * abs(m[-1]) + 2e-5 * np.abs(ref).max()
    assert err.max() <= 3 * omlp.inference_flip_bound(m) + noise, err.max()
    # almost every row carries no flip
    assert np.quantile(err, 0.98) <= noise


def test_features_match_oracle():
    Hm = make_hamiltonian(5, 17, 40, seed=8)
    h = b.ccsd_create(Hm.eps, Hm.h, Hm.B, Hm.o, Hm.v, Hm.naux)
    try:
        X = np.zeros((Hm.o ** 2 * Hm.v ** 2, 3), dtype=np.float32)
        b.ccsd_guess_features(h, X)
    finally:
        b.ccsd_destroy(h)
    ref = omlp.features(Hm).reshape(-1, 3)
    np.testing.assert_allclose(X, ref, rtol=3e-7, atol=1e-12)


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(1)
    n = 60000
    X = rng.normal(0.0, 1.0, (n, 3)).astype(np.float32)
    T = (0.5 * X[:, 0] * np.tanh(X[:, 1]) - 0.2 * X[:, 2] ** 2).astype(np.float32)
    model, loss = lg.train(X, T, steps=1500, batch=2048, lr=3e-3, seed=3)
    # target variance is 1 in the trained units: the fit explains almost all of it
    assert loss < 0.02
    loss_check, _ = b.ccsd_mlp_gradient(model, X, T)
    assert loss_check == pytest.approx(loss, rel=1e-4)
    out = np.zeros(n, dtype=np.float32)
    b.ccsd_mlp_predict(model, X, out)
    assert np.mean((out - T) ** 2) / np.mean(T ** 2) < 0.05


def _residual_max(h, dim):
    t = np.zeros(dim)
    b.ccsd_get_amplitudes(h, t)
    om = np.zeros(dim)
    b.ccsd_residual(h, t, om)
    return np.abs(om).max(), t


def test_learned_guess_gain_on_held_out_system():
    o, v, naux = 4, 24, 98
    train_systems = [make_hamiltonian(o, v, naux, seed=s) for s in range(100, 106)]
    opts = b.ccsd_default_options(tol_res=1e-7)
    X, T = lg.generate(train_systems, opts)
    model, loss = lg.train(X, T, steps=2000, batch=4096, lr=2e-3, seed=5)
    assert np.isfinite(loss)

    Hm = make_hamiltonian(o, v, naux, seed=200)
    dim = b.vector_dim(o, v)
    results = {}
    for name, mdl in (("mp2", None), ("learned", model)):
        h = b.ccsd_create(Hm.eps, Hm.h, Hm.B, o, v, naux, opts)
        try:
            start = lg.guess_doubles(h, o, v, mdl)
            b.ccsd_set_guess_model(h, mdl)
            e, iters = b.ccsd_solve_ground(h)
            res, t = _residual_max(h, dim)
        finally:
            b.ccsd_destroy(h)
        results[name] = dict(start=start, e=e, iters=iters, res=res, t=t)
    t2 = results["mp2"]["t"][o * v:].reshape(o, o, v, v)
    d_mp2 = np.linalg.norm(results["mp2"]["start"] - t2)
    d_learned = np.linalg.norm(results["learned"]["start"] - t2)
    # same converged-residual criterion, same solution
    for r in results.values():
        assert r["res"] < 1e-7
    assert results["learned"]["e"] == pytest.approx(results["mp2"]["e"], abs=1e-9)
    assert np.abs(results["learned"]["t"] - results["mp2"]["t"]).max() < 1e-6
    # The learned start is closer to the converged doubles.  On these synthetic
    # Hamiltonians the three per-element features explain only a few per cent of
    # the variance of t_CCSD - t_MP2 (the rest comes from sums over other
    # elements), so the gain is a few per cent of the starting error and the
    # DIIS iteration count moves by at most one.
    print(f"start error: first-order {d_mp2:.4e}, learned {d_learned:.4e}; iterations "
          f"{results['mp2']['iters']} -> {results['learned']['iters']}")
    assert d_learned < 0.99 * d_mp2, (d_learned, d_mp2)
    # the learned start never costs iterations
    assert results["learned"]["iters"] <= results["mp2"]["iters"]


def test_guess_targets_and_starts_are_the_library_arithmetic():
    """ccsd_guess_targets gives T = converged - start doubles and ccsd_guess_doubles the start
    (t_MP2 or -eta/D, plus a model's correction) in the library; checked on the host against
    the handle's own amplitudes, multipliers and the model's predictions."""
    o, v, naux = 3, 10, 20
    Hm = make_hamiltonian(o, v, naux, seed=300)
    n1, n2 = o * v, o * o * v * v
    h = b.ccsd_create(Hm.eps, Hm.h, Hm.B, o, v, naux, b.ccsd_default_options(tol_res=1e-10, tol_lin=1e-10))
    try:
        b.ccsd_solve_ground(h)
        t, lam = np.zeros(n1 + n2), np.zeros(n1 + n2)
        b.ccsd_get_amplitudes(h, t, lam)
        rng = np.random.default_rng(1)
        model = np.zeros(b.MLP_PARAMS, dtype=np.float32)
        model[:b.MLP_TRAINABLE] = rng.normal(0.0, 0.1, b.MLP_TRAINABLE)
        model[b.MLP_TRAINABLE + 3:b.MLP_TRAINABLE + 6] = 1.0
        model[b.MLP_TRAINABLE + 6] = 1e-3
        for which, conv in ((b.GUESS_AMPLITUDES, t), (b.GUESS_MULTIPLIERS, lam)):
            X = np.zeros((n2, 3), dtype=np.float32)
            T = np.zeros(n2, dtype=np.float32)
            b.ccsd_guess_targets(h, which, X, T)
            start = np.zeros(n2)
            b.ccsd_guess_doubles(h, which, None, start)
            # the start's doubles are the first feature (FP32) and T = converged - start
            assert np.abs(X[:, 0] - start).max() <= 1e-7 * np.abs(start).max()
            assert np.abs(T - (conv[n1:] - start)).max() <= 1e-6 * np.abs(conv[n1:]).max()
            d = np.zeros(n2, dtype=np.float32)
            b.ccsd_mlp_predict(model, X, d)
            corrected = np.zeros(n2)
            b.ccsd_guess_doubles(h, which, model, corrected)
            assert np.abs(corrected - (start + d)).max() <= 1e-7 * np.abs(start + d).max()
    finally:
        b.ccsd_destroy(h)


def test_learned_multiplier_start_on_held_out_system():
    """The multiplier network, trained on converged ground multipliers of the generator's
    systems, starts Lambda of a held-out system no farther from the solution than the Jacobi
    step, never with more iterations, and the converged multipliers are unchanged.  (On these
    synthetic Hamiltonians the correction lambda - (-eta/D) comes from sums over other elements
    that the three per-element features do not see: measured 0.2454 -> 0.2454, 9 -> 9.)"""
    o, v, naux = 4, 24, 98
    train_systems = [make_hamiltonian(o, v, naux, seed=s) for s in range(100, 106)]
    opts = b.ccsd_default_options(tol_res=1e-8, tol_lin=1e-7)
    X, T = lg.generate(train_systems, opts, which=b.GUESS_MULTIPLIERS)
    model, loss = lg.train(X, T, steps=2000, batch=4096, lr=2e-3, seed=6)
    assert np.isfinite(loss)
    Hm = make_hamiltonian(o, v, naux, seed=200)
    n1 = o * v
    out = {}
    for name, mdl in (("jacobi", None), ("learned", model)):
        h = b.ccsd_create(Hm.eps, Hm.h, Hm.B, o, v, naux, opts)
        try:
            b.ccsd_set_multiplier_guess_model(h, mdl)
            b.ccsd_solve_ground(h)
            start = lg.guess_doubles(h, o, v, mdl, which=b.GUESS_MULTIPLIERS)
            lam = np.zeros(b.vector_dim(o, v))
            b.ccsd_get_amplitudes(h, None, lam)
            out[name] = dict(start=start.ravel(), lam=lam, iters=b.ccsd_solve_iterations(h)["lambda"])
        finally:
            b.ccsd_destroy(h)
    l2 = out["jacobi"]["lam"][n1:]
    d_j = np.linalg.norm(out["jacobi"]["start"] - l2)
    d_l = np.linalg.norm(out["learned"]["start"] - l2)
    print(f"Lambda start error: Jacobi {d_j:.4e}, learned {d_l:.4e}; iterations "
          f"{out['jacobi']['iters']} -> {out['learned']['iters']}")
    assert d_l <= 1.001 * d_j
    assert out["learned"]["iters"] <= out["jacobi"]["iters"]
    assert np.abs(out["learned"]["lam"] - out["jacobi"]["lam"]).max() < 1e-5
