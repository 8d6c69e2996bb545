"""Pins for the oracle's circuit description (Sec. II-A, II-C; Eqs. 4-5)."""
import math

import numpy as np
import pytest

from oracle import circuit


@pytest.mark.parametrize("n,d", [(8, 1), (50, 2), (100, 4), (165, 6), (7, 6), (5, 0), (12, 11)])
def test_edge_count(n, d):
    # |G| = sum_i min(d, n-1-i) = n d - d (d+1) / 2 when d <= n-1
    E = circuit.edges(n, d)
    assert len(E) == sum(min(d, n - 1 - i) for i in range(n))
    if d <= n - 1:
        assert len(E) == n * d - d * (d + 1) // 2
    assert all(1 <= j - i <= d for i, j in E)


@pytest.mark.parametrize("n,d,expect", [(8, 1, 7), (50, 2, 145), (100, 4, 681), (165, 6, 1774)])
def test_op_counts(n, d, expect):
    ops = circuit.schedule(n, d)
    assert len(ops) == circuit.n_two_site_ops(n, d) == expect


@pytest.mark.parametrize("n,d", [(9, 1), (9, 3), (12, 5), (6, 5), (30, 6)])
def test_schedule_replay(n, d):
    """Replay the op list on a position->qubit table: every edge of G meets
    exactly once on adjacent positions, and all qubits return home."""
    pos = list(range(n))          # pos[p] = qubit at position p
    seen = []
    n_swaps = 0
    for op in circuit.schedule(n, d):
        p = op.p
        assert 0 <= p < n - 1
        if op.kind in (circuit.RXX, circuit.SWAP_RXX):
            assert sorted((pos[p], pos[p + 1])) == list(op.edge)
            seen.append(tuple(op.edge))
        if op.kind in (circuit.SWAP, circuit.SWAP_RXX):
            pos[p], pos[p + 1] = pos[p + 1], pos[p]
            n_swaps += 1
    assert pos == list(range(n))
    assert sorted(seen) == sorted(circuit.edges(n, d))
    # the paper's routing uses 2(k-1) SWAPs per Rxx at distance k; neighbouring
    # back-and-forth pairs cancel, leaving 2(k_i - 1) per block i
    assert n_swaps == sum(2 * (min(d, n - 1 - i) - 1) for i in range(n - 1) if min(d, n - 1 - i) > 0)


def test_gate_identities():
    X = np.array([[0, 1], [1, 0]])
    XX = np.kron(X, X)
    # Rxx at theta = pi/2 is the Pauli product up to the phase -i
    assert np.allclose(circuit.rxx_matrix(math.pi / 2), -1j * XX, atol=1e-15)
    S = circuit.swap_matrix()
    assert np.allclose(S @ S, np.eye(4))
    for th in (0.0, 0.3, -1.7, 2.9):
        R = circuit.rxx_matrix(th)
        assert np.allclose(R.conj().T @ R, np.eye(4), atol=1e-14)
        assert np.allclose(S @ R, R @ S, atol=1e-15)      # Rxx is symmetric in its qubits
    # SWAP maps |s t> to |t s>: |01> (index 1) -> |10> (index 2)
    e = np.zeros(4); e[1] = 1
    assert np.allclose(S @ e, np.eye(4)[2])


def test_angles():
    x = np.array([0.2, -0.5, 1.0, 3.0])
    g = 0.7
    assert np.allclose(circuit.z_phases(x, g), g * x)
    assert circuit.xx_angle(x, g, 0, 1) == pytest.approx(g * g * math.pi / 2 * 0.8 * 1.5)
    # a feature equal to 1 switches its Rxx terms off (Eq. 5)
    assert circuit.xx_angle(x, g, 2, 3) == 0.0
