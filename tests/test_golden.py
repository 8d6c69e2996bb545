"""The stored tiny-workload Gram (tests/golden/, written from the brute-force
statevector by tests/golden/make_golden.py) against the oracle's MPS path:
exact MPS simulation (no truncation at n=8) and the transfer sweep of Fig. 2
must reproduce the statevector kernel of Eq. 1 to rounding."""
import os

import numpy as np

import workloads
from oracle import mps, overlap, statevector

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_gram_statevector.txt")


def load_tiny_golden() -> np.ndarray:
    rows = np.loadtxt(GOLDEN, comments="#")
    i, j = rows[:, 0].astype(int), rows[:, 1].astype(int)
    K = np.zeros((64, 64))
    K[i, j] = rows[:, 2]
    K[j, i] = rows[:, 2]
    return K


def test_golden_file_is_complete():
    rows = np.loadtxt(GOLDEN, comments="#")
    assert rows.shape == (64 * 65 // 2, 3)
    K = load_tiny_golden()
    assert np.all(K >= 0) and np.all(K <= 1 + 1e-12)
    assert np.allclose(np.diag(K), 1.0, atol=1e-13, rtol=0)


def test_oracle_mps_path_reproduces_golden():
    w = workloads.tiny()
    Kg = load_tiny_golden()
    S = [mps.build_mps(x, w.d, w.reps, w.gamma, w.chi_max, w.eps).sites for x in w.X]
    K = overlap.gram(S)
    assert np.max(np.abs(K - Kg)) < 1e-13


def test_statevector_still_gives_golden():
    w = workloads.tiny()
    Kg = load_tiny_golden()
    idx = np.arange(0, 64, 9)
    K = statevector.gram(w.X[idx], w.d, w.reps, w.gamma)
    assert np.max(np.abs(K - Kg[np.ix_(idx, idx)])) < 1e-15
