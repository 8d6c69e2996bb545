"""Seeded synthetic inputs for the quantum-kernel Gram workloads.

This module only draws data: it holds none of the method's arithmetic (no
angles, gates, states or overlaps), so both the CPU oracle and the CUDA path
can take their inputs from here without sharing any computation.

The paper evaluates on the Elliptic Bitcoin data set (165 features, binary
labels, balanced subsamples, 80/20 split; Sec. III, Sec. III-B).  That data set
is not available here, so each workload below is a synthetic stand-in with the
same shape: feature count, sample count, label balance and split.  The five
workloads are:

  tiny   n=8,   d=1, r=2, gamma=0.5,  exact (no truncation), N=64,
         x ~ U[-1, 1], seed 0.
  c50    n=50,  d=2, r=2, gamma=0.3,  chi_max=64,  eps=1e-8, N=1000,
         x ~ N(0,1) clipped to [-2, 2], seed 2.
  c100   n=100, d=4, r=2, gamma=0.2,  chi_max=128, eps=1e-8,
         4 Gaussian clusters (labels {0,1} / {2,3}), 3200 train + 800 test,
         columns standardised on the train split, seed 3.
  c165   n=165, d=6, r=2, gamma=0.15, chi_max=128, eps=1e-8,
         correlated Gaussian with a random covariance, 6400 train + 1600 test,
         standardised on the train split, labels from a noisy linear rule
         split at the median, seed 4.
  surr   the c165 data, used by the learned surrogate (pairs drawn separately
         with their own seed).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: circuit parameters plus the data matrix."""

    name: str
    n: int            # qubits = features
    d: int            # interaction distance
    reps: int         # circuit repetitions r
    gamma: float      # kernel bandwidth
    chi_max: int      # bond-dimension cap
    eps: float        # truncation tolerance (discarded weight <= eps^2)
    X: np.ndarray     # (N, n) float64, row-major; train rows first
    y: np.ndarray     # (N,) int labels
    n_train: int      # rows [0, n_train) are the training split
    store: str = "c64"  # storage precision of the packed states
    extra: dict = field(default_factory=dict)

    @property
    def X_train(self) -> np.ndarray:
        return self.X[: self.n_train]

    @property
    def X_test(self) -> np.ndarray:
        return self.X[self.n_train:]


def tiny() -> Workload:
    rng = np.random.default_rng(0)
    X = rng.uniform(-1.0, 1.0, size=(64, 8))
    y = (np.arange(64) % 2).astype(np.int64)
    return Workload("tiny", 8, 1, 2, 0.5, 16, 0.0, np.ascontiguousarray(X), y, 64, store="c128")


def c50(N: int = 1000) -> Workload:
    rng = np.random.default_rng(2)
    X = np.clip(rng.standard_normal((N, 50)), -2.0, 2.0)
    y = (np.arange(N) % 2).astype(np.int64)
    return Workload("c50", 50, 2, 2, 0.3, 64, 1e-8, np.ascontiguousarray(X), y, N)


def c100(n_train: int = 3200, n_test: int = 800) -> Workload:
    rng = np.random.default_rng(3)
    n = 100
    centres = rng.normal(0.0, 1.5, size=(4, n))
    per = 1000
    pts = np.concatenate([centres[c] + rng.standard_normal((per, n)) for c in range(4)])
    lab = np.repeat(np.array([0, 0, 1, 1]), per)
    perm = rng.permutation(len(pts))
    pts, lab = pts[perm], lab[perm]
    tot = n_train + n_test
    pts, lab = pts[:tot], lab[:tot]
    mu = pts[:n_train].mean(0)
    sd = pts[:n_train].std(0)
    X = (pts - mu) / sd
    return Workload("c100", n, 4, 2, 0.2, 128, 1e-8, np.ascontiguousarray(X), lab.astype(np.int64), n_train)


def c165(n_train: int = 6400, n_test: int = 1600) -> Workload:
    rng = np.random.default_rng(4)
    n = 165
    A = rng.standard_normal((n, n))
    cov = A @ A.T / n + 0.1 * np.eye(n)
    L = np.linalg.cholesky(cov)
    tot = 8000
    raw = rng.standard_normal((tot, n)) @ L.T
    w = rng.standard_normal(n)
    score = raw @ w + 0.5 * rng.standard_normal(tot) * np.sqrt(w @ cov @ w)
    lab = (score > np.median(score)).astype(np.int64)
    mu = raw[:6400].mean(0)
    sd = raw[:6400].std(0)
    X = (raw - mu) / sd
    keep = np.concatenate([np.arange(min(n_train, 6400)), 6400 + np.arange(min(n_test, 1600))])
    return Workload("c165", n, 6, 2, 0.15, 128, 1e-8, np.ascontiguousarray(X[keep]), lab[keep],
                    min(n_train, 6400))


def surrogate_pairs(n_train: int, n_fit: int, n_cal: int, n_hold: int, seed: int = 5):
    """Disjoint random (i, j) pairs with i < j from the train-train triangle.

    Returns three int32 arrays of shape (P, 2) for fitting, calibration and
    held-out judging.  Pairs are drawn without replacement.
    """
    rng = np.random.default_rng(seed)
    total = n_fit + n_cal + n_hold
    n_tri = n_train * (n_train - 1) // 2
    if total > n_tri:
        raise ValueError("not enough distinct pairs")
    lin = rng.choice(n_tri, size=total, replace=False)
    # invert the row-major enumeration of the strict upper triangle
    rows = np.arange(n_train, dtype=np.int64)
    starts = rows * n_train - rows * (rows + 1) // 2
    i = np.searchsorted(starts, lin, side="right") - 1
    j = i + 1 + (lin - starts[i])
    pairs = np.stack([i, j], axis=1).astype(np.int32)
    return pairs[:n_fit], pairs[n_fit:n_fit + n_cal], pairs[n_fit + n_cal:]


def random_rows(n: int, N: int, seed: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """Plain uniform rows for small parity cases."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(lo, hi, size=(N, n)))


BY_NAME = {"tiny": tiny, "c50": c50, "c100": c100, "c165": c165}
