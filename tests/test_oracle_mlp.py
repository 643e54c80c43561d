"""Pins for the FP64 reference of the schedule network: central finite differences and the Adam formula."""
import numpy as np

import synth
from oracle import mlp


def _data(seed, B=64):
    rng_w = synth.normal(seed, 1, mlp.n_params()) * 0.3
    X = synth.normal(seed, 2, B * mlp.D_IN).reshape(B, mlp.D_IN)
    act = (synth.uniform(seed, 3, B) * mlp.A).astype(np.int64)
    tgt = synth.normal(seed, 4, B)
    return rng_w, X, act, tgt


def test_gradient_matches_central_differences():
    w, X, act, tgt = _data(7)
    _, g = mlp.grad(w, X, act, tgt)
    eps = 1e-6
    idx = np.linspace(0, len(w) - 1, 60).astype(int)
    for i in idx:
        wp = w.copy(); wp[i] += eps
        wm = w.copy(); wm[i] -= eps
        fd = (mlp.loss(wp, X, act, tgt) - mlp.loss(wm, X, act, tgt)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_untaken_outputs_get_no_gradient():
    w, X, act, tgt = _data(8)
    act[:] = 3
    _, g = mlp.grad(w, X, act, tgt)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(g)
    assert np.all(W3[np.arange(mlp.A) != 3] == 0.0) and np.all(b3[np.arange(mlp.A) != 3] == 0.0)


def test_adam_step_formula():
    w = np.array([1.0, -2.0]); g = np.array([0.5, -0.25])
    m = np.zeros(2); v = np.zeros(2)
    w1, m1, v1 = mlp.adam(w, g, m, v, 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, so the step is lr * sign(g) (up to eps)
    np.testing.assert_allclose(w1, w - 0.1 * np.sign(g), rtol=0, atol=1e-7)


def test_training_reduces_loss():
    w, X, act, tgt = _data(9, B=256)
    tgt = np.sin(X[:, 0]) + 0.5 * X[:, 1] * (act % 3 == 0)
    m = np.zeros_like(w); v = np.zeros_like(w)
    l0 = mlp.loss(w, X, act, tgt)
    for t in range(1, 301):
        _, g = mlp.grad(w, X, act, tgt)
        w, m, v = mlp.adam(w, g, m, v, t, lr=3e-3)
    assert mlp.loss(w, X, act, tgt) < 0.3 * l0
