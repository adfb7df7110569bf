"""FP64 oracle for the learned cost model (test infrastructure only).

The paper (Section 3.2) ranks fusion implementations with an additive
predictor, max(t_t, t_c), of pre-benchmarked routine times.  This project adds
a small learned model beside it: a 3-layer perceptron with ReLU activations

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  f = W3 h2 + b3,

trained with the mean squared error on log run time and the Adam update
(Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015,
Algorithm 1).  Everything here is plain numpy in float64 with the backward
pass written out from the chain rule.
"""

from __future__ import annotations

import numpy as np


def init_params(d_in: int, hidden: int, rng_vals) -> dict:
    """Deterministic init from a flat array of uniform [-1, 1) draws
    (He-uniform scaling); ``rng_vals`` must hold at least n_params values."""
    shapes = [("W1", (hidden, d_in)), ("b1", (hidden,)), ("W2", (hidden, hidden)),
              ("b2", (hidden,)), ("W3", (1, hidden)), ("b3", (1,))]
    out, k = {}, 0
    vals = np.asarray(rng_vals, dtype=np.float64)
    for name, shp in shapes:
        cnt = int(np.prod(shp))
        fan_in = shp[1] if len(shp) == 2 else 1
        scale = np.sqrt(6.0 / fan_in) if name.startswith("W") else 0.0
        out[name] = vals[k:k + cnt].reshape(shp) * scale
        k += cnt
    return out


def n_params(d_in: int, hidden: int) -> int:
    return hidden * d_in + hidden + hidden * hidden + hidden + hidden + 1


def forward(P: dict, X: np.ndarray):
    """Returns (f, cache).  X is (batch, d_in)."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    f = (h2 @ P["W3"].T + P["b3"])[:, 0]
    return f, (X, z1, h1, z2, h2)


def loss(P: dict, X, y) -> float:
    f, _ = forward(P, X)
    return float(np.mean((f - np.asarray(y, dtype=np.float64)) ** 2))


def grad(P: dict, X, y):
    """Analytic gradient of the mean squared error.  Returns (loss, grads)."""
    f, (X, z1, h1, z2, h2) = forward(P, X)
    y = np.asarray(y, dtype=np.float64)
    B = X.shape[0]
    df = 2.0 * (f - y) / B                      # dL/df, shape (B,)
    g = {}
    g["W3"] = df[None, :] @ h2                  # (1, H)
    g["b3"] = np.array([df.sum()])
    dh2 = df[:, None] * P["W3"]                 # (B, H)
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((f - y) ** 2)), g


def adam_step(P, G, M, V, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) in place; t counts from 1."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mh = M[k] / (1 - b1 ** t)
        vh = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
