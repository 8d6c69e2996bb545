"""Host-side classification step (Sec. III-B, Eq. 9): the SMO C-SVM on a
precomputed kernel against scikit-learn's SVC (LIBSVM), ROC AUC against its
definition, and the Gaussian kernel against its formula."""
import numpy as np
import pytest

from paper_2411_09336_gb300 import classify  # noqa: E402  (host module, no GPU calls)


def _data(n=160, m=6, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, m))
    y = (X[:, 0] + 0.5 * X[:, 1] ** 2 + 0.3 * rng.normal(size=n) > 0.4).astype(int)
    return X, y


def test_auc_matches_pairwise_definition():
    rng = np.random.default_rng(1)
    y = rng.integers(0, 2, 300)
    s = np.round(rng.normal(size=300), 1)  # ties included
    pos, neg = s[y == 1], s[y == 0]
    ref = np.mean((pos[:, None] > neg[None, :]) + 0.5 * (pos[:, None] == neg[None, :]))
    assert classify.roc_auc(y, s) == pytest.approx(ref, abs=1e-12)


def test_gaussian_kernel_formula():
    X, _ = _data(20)
    a = classify.gaussian_alpha(X)
    assert a == pytest.approx(1.0 / (X.shape[1] * X.var()))
    K = classify.gaussian_kernel(X, X[:5], a)
    ref = np.exp(-a * ((X[:, None, :] - X[None, :5, :]) ** 2).sum(-1))
    assert np.allclose(K, ref, atol=1e-13)


@pytest.mark.parametrize("C", [0.01, 0.5, 4.0])
def test_svm_matches_libsvm(C):
    svm = pytest.importorskip("sklearn.svm")
    X, y = _data()
    K = classify.gaussian_kernel(X, X, classify.gaussian_alpha(X))
    ours = classify.SVM(C=C).fit(K[:120, :120], y[:120])
    ref = svm.SVC(C=C, kernel="precomputed", tol=1e-3).fit(K[:120, :120], y[:120])
    f_ours = ours.decision_function(K[120:, :120])
    f_ref = ref.decision_function(K[120:, :120])
    assert np.max(np.abs(f_ours - f_ref)) <= 2e-2 * max(1.0, np.max(np.abs(f_ref)))
    assert classify.roc_auc(y[120:], f_ours) == pytest.approx(classify.roc_auc(y[120:], f_ref), abs=0.02)


def test_svm_separable_and_dual_feasible():
    X, y = _data(80, seed=3)
    K = X @ X.T + 1.0
    m = classify.SVM(C=10.0).fit(K, y)
    yy = np.where(y > 0, 1.0, -1.0)
    a = m.coef_ * yy
    assert np.all(a >= -1e-12) and np.all(a <= 10.0 + 1e-12)
    assert abs(np.sum(a * yy)) < 1e-9
