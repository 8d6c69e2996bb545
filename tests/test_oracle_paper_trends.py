"""Qualitative behaviour the paper reports, checked on the oracle with
synthetic features rescaled to (0, 2) as the paper prepares its data
(Sec. II-A).  These catch gross mistakes (a repetition not applied, the
routing dropping gates, truncation keeping too much) that a self-consistent
oracle could otherwise hide.

* Sec. III-A, Gram runtime breakdown: the d = 1, gamma = 0.1 ansatz on 165
  qubits keeps the bond dimension at about 2.
* Sec. III-A, Table I: the largest bond dimension grows with the
  interaction distance d (m = 100, r = 2, gamma = 1.0 there).
* Sec. III-B, depth study: more repetitions concentrate the kernel (the
  off-diagonal overlaps shrink).
"""
import numpy as np
import pytest

from oracle import mps, statevector


def rescaled(rows, cols, seed):
    X = np.random.default_rng(seed).standard_normal((rows, cols))
    lo, hi = X.min(0), X.max(0)
    return 2.0 * (X - lo) / (hi - lo)


def test_bond_dimension_about_two_at_d1_gamma_01():
    X = rescaled(20, 165, seed=0)
    dims = [mps.build_mps(x, 1, 2, 0.1, 128, 1e-8).bond_dims for x in X[:4]]
    interior = np.concatenate([np.asarray(b[1:-1]) for b in dims])
    assert 1.5 <= interior.mean() <= 2.5
    assert interior.max() <= 4


def test_largest_bond_dimension_grows_with_d():
    X = rescaled(4, 40, seed=3)
    largest = [np.mean([max(mps.build_mps(x, d, 2, 1.0, 1024, 1e-8).bond_dims) for x in X[:2]])
               for d in (1, 2, 3, 4)]
    assert all(a < b for a, b in zip(largest, largest[1:])), largest


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_depth_concentrates_the_kernel(seed):
    X = rescaled(12, 10, seed=seed)
    off = ~np.eye(12, dtype=bool)
    means = [statevector.gram(X, 1, r, 0.3)[off].mean() for r in (1, 2, 3, 4)]
    assert all(a > b for a, b in zip(means, means[1:])), means
    assert means[-1] < 0.1 * means[0]
