"""Writes the stored expected values under tests/golden/.  Calls only the
oracle (and the seeded input generators); nothing here runs the CUDA path.

    python tests/golden/make_golden.py

tiny_gram_statevector.txt: the 64 x 64 kernel K_ij = |<psi(x_i)|psi(x_j)>|^2
(Eq. 1) of the n=8, d=1, r=2, gamma=0.5 workload (64 vectors x ~ U[-1, 1],
seed 0), from the brute-force 256-amplitude statevector of Eqs. 2-5: one
line "i j K_ij" per pair i <= j, K_ij printed with 17 significant digits.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import statevector  # noqa: E402


def tiny_gram() -> np.ndarray:
    w = workloads.tiny()
    return statevector.gram(w.X, w.d, w.reps, w.gamma)


def main() -> None:
    K = tiny_gram()
    path = os.path.join(HERE, "tiny_gram_statevector.txt")
    with open(path, "w") as f:
        f.write("# K_ij of the n=8 d=1 r=2 gamma=0.5 workload (64 vectors, seed 0), i <= j\n")
        f.write("# brute-force statevector (Eqs. 1-5); written by tests/golden/make_golden.py\n")
        for i in range(K.shape[0]):
            for j in range(i, K.shape[1]):
                f.write(f"{i} {j} {K[i, j]:.17g}\n")


if __name__ == "__main__":
    main()
