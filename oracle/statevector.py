"""Brute-force statevector of |psi(x)> = U(x)|+>^m (Eqs. 2-5), small n only.

Amplitude index b = sum_k b_k 2^(n-1-k): qubit 0 is the most significant bit,
so the vector reshaped to (2,)*n has qubit k on axis k.  Every Rxx of G is
applied directly on its two qubits (no routing, no truncation): this is the
definition, against which the MPS simulation is checked.
"""
from __future__ import annotations

import math

import numpy as np

from . import circuit


def state(x: np.ndarray, d: int, reps: int, gamma: float) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if n > 16:
        raise ValueError("statevector oracle is for n <= 16")
    psi = np.full((2,) * n, 2.0 ** (-n / 2.0), dtype=np.complex128)  # |+>^n, Eq. 2
    phi = circuit.z_phases(x, gamma)
    for _ in range(reps):
        # exp(-i H_Z): qubit k contributes exp(-i phi_k z_k), z = +1 for |0>, -1 for |1>
        for k in range(n):
            shape = [1] * n
            shape[k] = 2
            psi = psi * np.exp(-1j * phi[k] * np.array([1.0, -1.0])).reshape(shape)
        # exp(-i H_XX) = prod over edges of (cos th I - i sin th X_i X_j); the terms commute
        for (i, j) in circuit.edges(n, d):
            th = circuit.xx_angle(x, gamma, i, j)
            flipped = np.flip(np.flip(psi, axis=i), axis=j)
            psi = math.cos(th) * psi - 1j * math.sin(th) * flipped
    return psi.reshape(-1)


def gram(X: np.ndarray, d: int, reps: int, gamma: float, Y: np.ndarray | None = None) -> np.ndarray:
    """K_ij = |<psi(x_i)|psi(y_j)>|^2 (Eq. 1) from explicit statevectors."""
    SA = np.stack([state(x, d, reps, gamma) for x in X])
    SB = SA if Y is None else np.stack([state(y, d, reps, gamma) for y in Y])
    Z = SA.conj() @ SB.T
    return np.abs(Z) ** 2
