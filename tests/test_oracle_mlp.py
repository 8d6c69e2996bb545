"""Pins for the surrogate MLP oracle: finite differences, closed-form cases,
Adam's first-step property and split-conformal coverage."""
import math

import numpy as np
import pytest

from oracle import mlp


def small_net(seed=0, din=6, h=5):
    rng = np.random.default_rng(seed)
    P = mlp.init_params(din, h, rng)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0, 0.1, P[k].shape)
    F = rng.normal(0, 1, (9, din))
    t = rng.normal(0, 1, 9)
    return P, F, t


def test_gradients_finite_difference():
    P, F, t = small_net()
    L, g = mlp.loss_and_grads(P, F, t)
    h = 1e-6
    for k in P:
        it = np.nditer(P[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            fd = (mlp.loss_and_grads(Pp, F, t)[0] - mlp.loss_and_grads(Pm, F, t)[0]) / (2 * h)
            assert g[k][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, idx)


def test_constant_output_case():
    """W3 = 0: the net outputs b3 everywhere and dL/db3 = mean(b3 - t)."""
    P, F, t = small_net(1)
    P["W3"][:] = 0.0
    y, _ = mlp.forward(P, F)
    assert np.allclose(y, P["b3"][0])
    L, g = mlp.loss_and_grads(P, F, t)
    assert L == pytest.approx(0.5 * np.mean((P["b3"][0] - t) ** 2))
    assert g["b3"][0] == pytest.approx(np.mean(P["b3"][0] - t))
    assert np.allclose(g["W1"], 0) and np.allclose(g["W2"], 0)


def test_adam_first_step_is_signed_lr():
    """After one step from zero moments the bias-corrected update is
    lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps."""
    P, F, t = small_net(2)
    _, g = mlp.loss_and_grads(P, F, t)
    m = {k: np.zeros_like(v) for k, v in P.items()}
    v = {k: np.zeros_like(v) for k, v in P.items()}
    P0 = {k: x.copy() for k, x in P.items()}
    mlp.adam_step(P, g, m, v, 1, 1e-3)
    for k in P:
        want = P0[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(P[k], want, rtol=0, atol=1e-12)


def test_pair_features_symmetric():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, 4))
    pr = np.array([[0, 1], [2, 5], [3, 3]])
    f1 = mlp.pair_features(X, X, pr)
    f2 = mlp.pair_features(X, X, pr[:, ::-1])
    assert np.array_equal(f1, f2)
    assert f1.shape == (3, 8)
    assert np.allclose(f1[2, :4], 0)


def test_pair_features_by_hand():
    """x = (1, 2), y = (3, 5): squared differences (4, 9), midpoints (2, 3.5);
    a pair of a point with itself gives (0, 0, x)."""
    Xa = np.array([[1.0, 2.0]])
    Xb = np.array([[3.0, 5.0], [1.0, 2.0]])
    f = mlp.pair_features(Xa, Xb, np.array([[0, 0], [0, 1]]))
    assert np.array_equal(f, np.array([[4.0, 9.0, 2.0, 3.5], [0.0, 0.0, 1.0, 2.0]]))


def test_conformal_coverage():
    """For exchangeable residuals the split-conformal bound covers a fresh
    point with probability >= 1 - alpha."""
    rng = np.random.default_rng(4)
    alpha = 0.1
    hits = []
    for trial in range(200):
        pred = rng.uniform(0, 1, 101)
        truth = pred + rng.normal(0, 0.2, 101)
        b = mlp.conformal_bounds(pred[:100], truth[:100], np.array([0.0, 1.0 + 1e-12]), alpha)
        hits.append(abs(pred[100] - truth[100]) <= b[0])
    assert np.mean(hits) >= 1 - alpha - 0.05
    # a Gaussian residual's 90% two-sided bound is 1.645 sigma
    pred = np.zeros(100000); truth = rng.normal(0, 1, 100000)
    b = mlp.conformal_bounds(pred, truth, np.array([-1.0, 1.0]), 0.1)
    assert b[0] == pytest.approx(1.645, rel=0.02)
    # an empty bin has no bound
    b = mlp.conformal_bounds(pred, truth, np.array([-1.0, 1.0, 2.0]), 0.1)
    assert math.isinf(b[1])
