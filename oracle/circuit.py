"""Feature-map circuit of Sec. II-A / II-C: edge set, angles and op schedule.

U(x) = (exp(-i H_XX) exp(-i H_Z))^r applied to |+>^m (Eqs. 2-3) with
  H_Z  = gamma * sum_k x_k Z_k                                  (Eq. 4)
  H_XX = gamma^2 (pi/2) sum_{(i,j) in G} (1-x_i)(1-x_j) X_i X_j (Eq. 5)
G is the linear chain with every pair at distance 1..d (Sec. II-C).

Readings used here (shared by every implementation of the method):
  * The features are used as given (no (0,2) rescaling inside the method).
  * exp(-i phi Z) with phi = gamma*x_k gives |0> -> e^{-i phi}|0>,
    |1> -> e^{+i phi}|1>; exp(-i theta XX) = cos(theta) I - i sin(theta) XX.
  * Within one repetition the Z layer comes first, then every Rxx of G.
  * Rxx on (i, i+t), t > 1, is routed by SWAPs (Sec. II-C: t-1 SWAPs before
    and after).  Walking qubit i to the right through its block
    {(i,i+1), ..., (i,i+k)} and back, the back-to-back SWAP pairs of
    neighbouring gates cancel, leaving per block i (k = min(d, n-1-i)):
       for t = 1..k-1 : Rxx(i, i+t) then SWAP, on positions (i+t-1, i+t)
       t = k          : Rxx(i, i+k) on positions (i+k-1, i+k)
       back           : SWAP on positions (i+k-2, i+k-1), ..., (i, i+1)
    i.e. 2k-1 two-site ops, each applied (and truncated) as one 2-site gate.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# op kinds
RXX = 0        # Rxx(theta) on the adjacent pair
SWAP_RXX = 1   # SWAP after Rxx(theta) (the two commute)
SWAP = 2       # bare SWAP


@dataclass(frozen=True)
class Op:
    kind: int
    p: int            # the op acts on MPS positions (p, p+1)
    edge: tuple       # (i, j) qubit pair of the Rxx angle, or None


def edges(n: int, d: int) -> list[tuple[int, int]]:
    """Edge set G: all (i, j) with 1 <= j - i <= d (Sec. II-C)."""
    return [(i, j) for i in range(n) for j in range(i + 1, min(n, i + d + 1))]


def z_phases(x: np.ndarray, gamma: float) -> np.ndarray:
    """phi_k = gamma * x_k, the Rz phase of Eq. 4."""
    return gamma * np.asarray(x, dtype=np.float64)


def xx_angle(x: np.ndarray, gamma: float, i: int, j: int) -> float:
    """theta_ij = gamma^2 (pi/2) (1 - x_i)(1 - x_j), the coefficient of Eq. 5."""
    return gamma * gamma * (math.pi / 2.0) * (1.0 - x[i]) * (1.0 - x[j])


def schedule(n: int, d: int) -> list[Op]:
    """Two-site op list for one repetition of exp(-i H_XX) (routing above)."""
    ops: list[Op] = []
    for i in range(n - 1):
        k = min(d, n - 1 - i)
        if k <= 0:
            continue
        for t in range(1, k):
            ops.append(Op(SWAP_RXX, i + t - 1, (i, i + t)))
        ops.append(Op(RXX, i + k - 1, (i, i + k)))
        for p in range(i + k - 2, i - 1, -1):
            ops.append(Op(SWAP, p, None))
    return ops


def n_two_site_ops(n: int, d: int) -> int:
    """sum_i (2 k_i - 1), k_i = min(d, n-1-i): the count the schedule must have."""
    return sum(2 * min(d, n - 1 - i) - 1 for i in range(n - 1) if min(d, n - 1 - i) > 0)


def rxx_matrix(theta: float) -> np.ndarray:
    """exp(-i theta X (x) X) in the basis |s t>, index 2*s + t."""
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    return math.cos(theta) * np.eye(4) - 1j * math.sin(theta) * np.kron(X, X)


def swap_matrix() -> np.ndarray:
    S = np.zeros((4, 4))
    for s in range(2):
        for t in range(2):
            S[2 * t + s, 2 * s + t] = 1.0
    return S


def op_matrix(op: Op, x: np.ndarray, gamma: float) -> np.ndarray:
    """4x4 gate of one scheduled op (rows/cols index 2*s + t)."""
    if op.kind == SWAP:
        return swap_matrix().astype(np.complex128)
    g = rxx_matrix(xx_angle(x, gamma, *op.edge))
    if op.kind == SWAP_RXX:
        g = swap_matrix() @ g
    return g
