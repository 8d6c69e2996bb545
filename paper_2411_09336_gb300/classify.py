"""Kernel SVM on a precomputed Gram matrix, ROC AUC, and the Gaussian-kernel
baseline: the classification step that consumes the quantum kernel
(Sec. III-B; Eq. 9 defines the Gaussian kernel the paper compares with).

Host code (numpy): the Gram matrices come from qk_gram; nothing here touches
the GPU.  The solver is sequential minimal optimisation for the C-SVM dual

    max_a  sum_i a_i - 1/2 sum_ij a_i a_j y_i y_j K_ij,
    0 <= a_i <= C,  sum_i a_i y_i = 0,

with the working-set selection of Fan, Chen and Lin (JMLR 6, 2005): the
maximal violating i, and j by the second-order gain, stopping when the
violation m(a) - M(a) <= tol (the criterion of LIBSVM and scikit-learn's
SVC, tol = 1e-3 by default).
"""
from __future__ import annotations

import numpy as np

__all__ = ["SVM", "roc_auc", "gaussian_kernel", "gaussian_alpha"]


class SVM:
    """C-SVM with a precomputed kernel.  Labels in {0, 1} or {-1, +1}."""

    def __init__(self, C: float = 1.0, tol: float = 1e-3, max_iter: int = 1_000_000):
        if not C > 0:
            raise ValueError("C must be positive")
        self.C, self.tol, self.max_iter = float(C), float(tol), int(max_iter)

    def fit(self, K: np.ndarray, y: np.ndarray) -> "SVM":
        K = np.asarray(K, dtype=np.float64)
        y = np.where(np.asarray(y) > 0, 1.0, -1.0)
        n = len(y)
        if K.shape != (n, n):
            raise ValueError("K must be n x n")
        C, tau = self.C, 1e-12
        Q = K * np.outer(y, y)
        a = np.zeros(n)
        G = -np.ones(n)                      # gradient of the dual objective (minimised)
        diag = np.diag(Q).copy()
        it = 0
        for it in range(self.max_iter):
            # I_up: y=+1, a<C or y=-1, a>0 ; I_low: y=+1, a>0 or y=-1, a<C
            up = ((y > 0) & (a < C)) | ((y < 0) & (a > 0))
            low = ((y > 0) & (a > 0)) | ((y < 0) & (a < C))
            v = -y * G
            if not up.any() or not low.any():
                break
            i = int(np.argmax(np.where(up, v, -np.inf)))
            m_up = v[i]
            m_low = np.min(np.where(low, v, np.inf))
            if m_up - m_low <= self.tol:
                break
            # second-order choice of j among I_low with v_j < v_i
            b = m_up - v
            cand = low & (b > 0)
            aij = diag[i] + diag - 2.0 * y[i] * y * Q[i]  # K_ii + K_jj - 2 K_ij (Q_ij = y_i y_j K_ij)
            aij = np.where(aij > 0, aij, tau)
            gain = np.where(cand, -(b * b) / aij, np.inf)
            j = int(np.argmin(gain))
            # update the pair (two-variable subproblem, clipped to the box)
            yi, yj = y[i], y[j]
            Kij = K[i, j]
            quad = K[i, i] + K[j, j] - 2.0 * Kij
            quad = quad if quad > 0 else tau
            ai_old, aj_old = a[i], a[j]
            if yi != yj:
                delta = (-G[i] - G[j]) / quad
                diff = ai_old - aj_old
                ai, aj = ai_old + delta, aj_old + delta
                if diff > 0:
                    if aj < 0:
                        aj, ai = 0.0, diff
                else:
                    if ai < 0:
                        ai, aj = 0.0, -diff
                if diff > 0:
                    if ai > C:
                        ai, aj = C, C - diff
                else:
                    if aj > C:
                        aj, ai = C, C + diff
            else:
                delta = (G[i] - G[j]) / quad
                s = ai_old + aj_old
                ai, aj = ai_old - delta, aj_old + delta
                if s > C:
                    if ai > C:
                        ai, aj = C, s - C
                else:
                    if aj < 0:
                        aj, ai = 0.0, s
                if s > C:
                    if aj > C:
                        aj, ai = C, s - C
                else:
                    if ai < 0:
                        ai, aj = 0.0, s
            da, db = ai - ai_old, aj - aj_old
            a[i], a[j] = ai, aj
            G += Q[:, i] * da + Q[:, j] * db
        self.n_iter_ = it
        # offset rho (decision = sum_i a_i y_i K(x_i, x) - rho): the mean of
        # y_i G_i over free vectors, else the midpoint of its feasible interval
        yG = y * G
        free = (a > 0) & (a < C)
        if free.any():
            rho = float(np.mean(yG[free]))
        else:
            ub_set = ((a >= C) & (y < 0)) | ((a <= 0) & (y > 0))
            lb_set = ((a >= C) & (y > 0)) | ((a <= 0) & (y < 0))
            ub = np.min(yG[ub_set]) if ub_set.any() else np.inf
            lb = np.max(yG[lb_set]) if lb_set.any() else -np.inf
            rho = 0.5 * (ub + lb)
        self.coef_ = a * y
        self.intercept_ = -rho
        self.support_ = np.nonzero(a > 0)[0]
        return self

    def decision_function(self, K_test_train: np.ndarray) -> np.ndarray:
        """Scores for rows of K(test, train); positive means class 1."""
        return np.asarray(K_test_train, dtype=np.float64) @ self.coef_ + self.intercept_


def roc_auc(y: np.ndarray, scores: np.ndarray) -> float:
    """Area under the ROC curve: the probability that a random positive
    scores above a random negative (ties count one half)."""
    y = np.asarray(y) > 0
    s = np.asarray(scores, dtype=np.float64)
    pos, neg = s[y], s[~y]
    if len(pos) == 0 or len(neg) == 0:
        raise ValueError("both classes are needed")
    order = np.argsort(np.concatenate([pos, neg]), kind="mergesort")
    allv = np.concatenate([pos, neg])[order]
    # average ranks over ties
    ranks = np.empty(len(allv))
    i = 0
    while i < len(allv):
        j = i
        while j + 1 < len(allv) and allv[j + 1] == allv[i]:
            j += 1
        ranks[i:j + 1] = 0.5 * (i + j) + 1.0
        i = j + 1
    r = np.empty(len(allv))
    r[order] = ranks
    r_pos = r[:len(pos)].sum()
    return float((r_pos - len(pos) * (len(pos) + 1) / 2.0) / (len(pos) * len(neg)))


def gaussian_alpha(X: np.ndarray) -> float:
    """The Gaussian kernel's width of Eq. 9: alpha = 1 / (m Var(X)), m the
    number of features and Var the variance of all training entries."""
    X = np.asarray(X, dtype=np.float64)
    return 1.0 / (X.shape[1] * X.var())


def gaussian_kernel(X1: np.ndarray, X2: np.ndarray, alpha: float) -> np.ndarray:
    """k(x, y) = exp(-alpha ||x - y||^2) (Eq. 9)."""
    X1, X2 = np.asarray(X1, dtype=np.float64), np.asarray(X2, dtype=np.float64)
    d2 = (np.sum(X1 * X1, 1)[:, None] + np.sum(X2 * X2, 1)[None, :] - 2.0 * X1 @ X2.T)
    return np.exp(-alpha * np.maximum(d2, 0.0))
