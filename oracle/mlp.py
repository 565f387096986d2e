"""The rank predictor's network in FP64 (oracle; test infrastructure).

A multilayer perceptron 16 -> 64 -> 64 -> 1 with ReLU activations maps the
geometry features of a cluster to the fraction k / n of its dimension that
the rank-revealing compression keeps (the learned rank of the north-star
extension to Algorithm 1; the paper has no counterpart).  Parameters, in the
flat order the library's C ABI uses:

    W1 (64 x 16, row-major), b1 (64), W2 (64 x 64, row-major), b2 (64),
    w3 (64), b3 (1)                                  -> 5313 numbers

Forward:  z1 = W1 x + b1,  h1 = max(z1, 0),  z2 = W2 h1 + b2,
          h2 = max(z2, 0),  o = w3 . h2 + b3.
Loss:     mean over the batch of (o - y)^2.
Gradients by the chain rule (written out below, one line per step; the
derivative of max(z, 0) is taken as 1 for z > 0 and 0 otherwise).

Every step is plain NumPy in FP64; the tests pin it against central finite
differences of the loss.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 16, 64
SHAPES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("w3", (N_HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    """Split the flat parameter vector into the named arrays (views)."""
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Network output o for every row of X (n x 16)."""
    p = unpack(theta)
    h1 = np.maximum(X @ p["W1"].T + p["b1"], 0.0)
    h2 = np.maximum(h1 @ p["W2"].T + p["b2"], 0.0)
    return h2 @ p["w3"] + p["b3"][0]


def loss_and_grad(theta: np.ndarray, X: np.ndarray, y: np.ndarray):
    """Mean squared error over the batch and its gradient (flat, FP64)."""
    p = unpack(theta)
    n = X.shape[0]
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["w3"] + p["b3"][0]
    e = o - y
    loss = float(np.mean(e * e))
    do = 2.0 * e / n                       # d loss / d o
    g = {"w3": h2.T @ do, "b3": np.array([do.sum()])}
    dz2 = np.outer(do, p["w3"]) * (z2 > 0)  # d loss / d z2
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)        # d loss / d z1
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)
