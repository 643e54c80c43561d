"""FP64 reference of the restart-schedule network: forward, loss, gradient.

TEST INFRASTRUCTURE ONLY (the oracle of the CUDA kernels in eik_mlp.cu).  The
schedule network has no counterpart in the paper; it picks the stride and block
edge of each restart of Alg. 6 from front statistics, and only changes which
restart does which work, never the solution.

Network: x (D_IN) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> W3 h2 + b3 (A),
one output per action (a predicted log cost rate).  Parameters are one flat
vector in the order W1 (H x D_IN, row-major), b1, W2 (H x H), b2, W3 (A x H), b3.
Loss over a batch: mean_s (y_s[a_s] - t_s)^2, the squared error of the taken
action's output only.
"""
from __future__ import annotations

import numpy as np

D_IN = 10
H = 32
A = 12


def n_params(d_in: int = D_IN, h: int = H, a: int = A) -> int:
    return h * d_in + h + h * h + h + a * h + a


def unpack(w: np.ndarray, d_in: int = D_IN, h: int = H, a: int = A):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + h * d_in].reshape(h, d_in); o += h * d_in
    b1 = w[o:o + h]; o += h
    W2 = w[o:o + h * h].reshape(h, h); o += h * h
    b2 = w[o:o + h]; o += h
    W3 = w[o:o + a * h].reshape(a, h); o += a * h
    b3 = w[o:o + a]; o += a
    return W1, b1, W2, b2, W3, b3


def forward(w: np.ndarray, X: np.ndarray):
    """Outputs (B, A) and the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, h1, h2


def loss(w: np.ndarray, X: np.ndarray, act: np.ndarray, tgt: np.ndarray) -> float:
    Y, _, _ = forward(w, X)
    e = Y[np.arange(len(act)), act] - tgt
    return float(np.mean(e * e))


def grad(w: np.ndarray, X: np.ndarray, act: np.ndarray, tgt: np.ndarray):
    """(loss, d loss / d w) by the chain rule, layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    B = len(act)
    Y, h1, h2 = forward(w, X)
    e = Y[np.arange(B), act] - tgt
    dY = np.zeros_like(Y)
    dY[np.arange(B), act] = 2.0 * e / B
    gW3 = dY.T @ h2
    gb3 = dY.sum(0)
    dh2 = (dY @ W3) * (1.0 - h2 * h2)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (1.0 - h1 * h1)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(np.mean(e * e)), g


def adam(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015); returns the new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
