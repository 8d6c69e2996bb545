"""MPS inner products and the Gram matrix (Eq. 1, Fig. 2).

z = <psi_a|psi_b> is contracted site by site from the left (Fig. 2): the bra
tensors are conjugated, both states are joined on their qubit legs, and the
running environment E (chi^a_k x chi^b_k) absorbs one site pair per step:
    E_0 = [[1]],   E_{k+1} = sum_s A_k[:, s, :]^dagger E_k B_k[:, s, :],
    z = E_n[0, 0],  K = |z|^2.
sweep_right_to_left contracts the same network from the other end and serves
as an independent cross-check.
"""
from __future__ import annotations

import numpy as np


def sweep_left_to_right(A, B) -> complex:
    E = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        T = np.tensordot(E, b, axes=(1, 0))                       # (chiA_k, 2, chiB_k+1)
        E = np.tensordot(a.conj(), T, axes=([0, 1], [0, 1]))     # (chiA_k+1, chiB_k+1)
    return complex(E[0, 0])


def sweep_right_to_left(A, B) -> complex:
    F = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(reversed(A), reversed(B)):
        T = np.tensordot(b, F, axes=(2, 1))                       # (chiB_k, 2, chiA_k+1)
        F = np.tensordot(a.conj(), T, axes=([1, 2], [1, 2]))      # (chiA_k, chiB_k)
    return complex(F[0, 0])


def kernel_entry(A, B) -> float:
    z = sweep_left_to_right(A, B)
    return abs(z) ** 2


def gram(states_a, states_b=None) -> np.ndarray:
    """K_ij = |<psi_i|psi_j>|^2 (Eq. 1).  states_b None: the symmetric case,
    computed for i <= j and mirrored (Sec. II-D)."""
    sym = states_b is None
    sb = states_a if sym else states_b
    K = np.zeros((len(states_a), len(sb)))
    for i, A in enumerate(states_a):
        for j in range(i if sym else 0, len(sb)):
            K[i, j] = kernel_entry(A, sb[j])
            if sym:
                K[j, i] = K[i, j]
    return K


def product_state_kernel(x, y, reps: int, gamma: float) -> float:
    """d = 0 closed form: each qubit ends in (e^{-i r g x}|0> + e^{i r g x}|1>)/sqrt 2,
    so K = prod_k cos^2(r gamma (x_k - y_k))  (Eqs. 1, 2, 4 with G empty)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.prod(np.cos(reps * gamma * (x - y)) ** 2))
