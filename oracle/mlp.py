"""MLP surrogate for log K (not in the paper; FP64 reference of its arithmetic).

Network: f -> ReLU(W1 f + b1) -> ReLU(W2 h1 + b2) -> w3 . h2 + b3.
Pair features (symmetric in the two data vectors, so the prediction is too):
    f(x, y) = [ (x - y)^2 , (x + y) / 2 ]          (2n values)
Loss: L = (1 / 2P) sum_p (yhat_p - t_p)^2 over a batch of P pairs.
Optimiser: Adam (Kingma & Ba 2015), bias-corrected moments.
Calibration: split conformal; per bin of predicted value, the bound is the
ceil((m+1)(1-alpha))-th smallest absolute residual of the m calibration
points in that bin (Vovk et al.; Lei et al. 2018).

Weights are stored as W[out, in] row-major.
"""
from __future__ import annotations

import math

import numpy as np


def pair_features(Xa: np.ndarray, Xb: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    a = Xa[pairs[:, 0]]
    b = Xb[pairs[:, 1]]
    return np.concatenate([(a - b) ** 2, 0.5 * (a + b)], axis=1)


def init_params(in_dim: int, hidden: int, rng: np.random.Generator) -> dict:
    """He-uniform init for the ReLU layers, zero biases."""
    def he(o, i):
        lim = math.sqrt(6.0 / i)
        return rng.uniform(-lim, lim, size=(o, i))
    return {"W1": he(hidden, in_dim), "b1": np.zeros(hidden),
            "W2": he(hidden, hidden), "b2": np.zeros(hidden),
            "W3": he(1, hidden), "b3": np.zeros(1)}


def forward(P: dict, F: np.ndarray):
    z1 = F @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["W3"].T + P["b3"]
    return y[:, 0], (F, z1, h1, z2, h2)


def loss_and_grads(P: dict, F: np.ndarray, t: np.ndarray):
    y, (F, z1, h1, z2, h2) = forward(P, F)
    n = len(t)
    r = y - t
    L = 0.5 * float(np.mean(r * r))
    dy = (r / n)[:, None]                     # dL/dy
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(0)
    dh2 = dy @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ F
    g["b1"] = dz1.sum(0)
    return L, g


def adam_step(P: dict, g: dict, m: dict, v: dict, step: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; step counts from 1."""
    for k in P:
        m[k] = b1 * m[k] + (1.0 - b1) * g[k]
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k]
        mh = m[k] / (1.0 - b1 ** step)
        vh = v[k] / (1.0 - b2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def conformal_bounds(pred: np.ndarray, truth: np.ndarray, edges: np.ndarray, alpha: float) -> np.ndarray:
    """Per-bin split-conformal bound on |pred - truth|; bins are [edges[b], edges[b+1]).
    A bin with too few points for the requested coverage gets +inf."""
    res = np.abs(pred - truth)
    nb = len(edges) - 1
    out = np.full(nb, np.inf)
    idx = np.clip(np.searchsorted(edges, pred, side="right") - 1, 0, nb - 1)
    for b in range(nb):
        rb = np.sort(res[idx == b])
        m = len(rb)
        q = math.ceil((m + 1) * (1.0 - alpha))
        if m > 0 and q <= m:
            out[b] = rb[q - 1]
    return out
