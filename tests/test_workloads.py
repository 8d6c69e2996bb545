"""The synthetic inputs follow their stated recipes (shapes, seeds, value
ranges, standardisation on the train split, label balance) and the pair
sampler's inversion of the upper-triangle enumeration is exact."""
import numpy as np

import workloads


def test_tiny_recipe():
    w = workloads.tiny()
    assert w.X.shape == (64, 8) and (w.n, w.d, w.reps, w.gamma, w.eps) == (8, 1, 2, 0.5, 0.0)
    assert np.array_equal(w.X, np.random.default_rng(0).uniform(-1.0, 1.0, size=(64, 8)))
    assert w.X.min() >= -1.0 and w.X.max() <= 1.0


def test_c50_recipe():
    w = workloads.c50()
    assert w.X.shape == (1000, 50) and (w.d, w.reps, w.gamma, w.chi_max, w.eps) == (2, 2, 0.3, 64, 1e-8)
    assert w.X.min() >= -2.0 and w.X.max() <= 2.0
    assert np.mean(np.abs(w.X) == 2.0) > 0.01        # clipping happened
    assert np.array_equal(workloads.c50(N=40).X, w.X[:40])


def test_c100_recipe():
    w = workloads.c100()
    assert w.X.shape == (4000, 100) and w.n_train == 3200 and w.X_test.shape == (800, 100)
    assert np.allclose(w.X_train.mean(0), 0.0, atol=1e-12)
    assert np.allclose(w.X_train.std(0), 1.0, atol=1e-12)
    assert abs(w.y.mean() - 0.5) < 0.05 and set(np.unique(w.y)) == {0, 1}


def test_c165_recipe():
    w = workloads.c165()
    assert w.X.shape == (8000, 165) and w.n_train == 6400
    assert (w.d, w.reps, w.gamma, w.chi_max, w.eps) == (6, 2, 0.15, 128, 1e-8)
    assert np.allclose(w.X_train.mean(0), 0.0, atol=1e-12)
    assert np.allclose(w.X_train.std(0), 1.0, atol=1e-12)
    assert abs(w.y.mean() - 0.5) < 0.01              # split at the median
    # correlated features (random covariance): the mean |correlation| is
    # about 3x that of independent columns of the same length (~0.018)
    C = np.corrcoef(w.X_train[:2000].T)
    assert np.abs(C[np.triu_indices(165, 1)]).mean() > 0.04
    small = workloads.c165(n_train=100, n_test=10)
    assert np.array_equal(small.X[:100], w.X[:100]) and np.array_equal(small.X[100:], w.X[6400:6410])


def test_surrogate_pairs_disjoint_and_in_triangle():
    n = 37
    fit, cal, hold = workloads.surrogate_pairs(n, 300, 100, 100, seed=1)
    allp = np.concatenate([fit, cal, hold])
    assert allp.shape == (500, 2)
    assert np.all(allp[:, 0] < allp[:, 1]) and allp.min() >= 0 and allp.max() < n
    assert len({(int(i), int(j)) for i, j in allp}) == 500
    # every pair of a tiny triangle is reachable: draw all of them
    f, c, h = workloads.surrogate_pairs(5, 10, 0, 0, seed=2)
    assert sorted(map(tuple, f.tolist())) == [(i, j) for i in range(5) for j in range(i + 1, 5)]
