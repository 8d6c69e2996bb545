"""Pins for the oracle's statevector, MPS simulation and overlaps.

Everything here is checked against something other than the code under
test: the d = 0 closed form, a hand-expanded two-qubit state, gate algebra,
the brute-force statevector (for the MPS), the second sweep order (for the
overlap), canonical-form identities and the truncation bound of Eq. 8.
"""
import math

import numpy as np
import pytest

from oracle import circuit, mps, overlap, statevector


def test_two_qubit_state_by_hand():
    """n=2, d=1, r=1: U|++> written out amplitude by amplitude (Eqs. 2-5)."""
    x = np.array([0.3, -0.8]); g = 0.9
    p0, p1 = g * x
    th = g * g * math.pi / 2 * (1 - x[0]) * (1 - x[1])
    amp = {}
    for s in (0, 1):
        for t in (0, 1):
            amp[(s, t)] = 0.5 * np.exp(-1j * p0 * (1 - 2 * s)) * np.exp(-1j * p1 * (1 - 2 * t))
    want = np.array([math.cos(th) * amp[(s, t)] - 1j * math.sin(th) * amp[(1 - s, 1 - t)]
                     for s in (0, 1) for t in (0, 1)])
    got = statevector.state(x, 1, 1, g)
    assert np.allclose(got, want, atol=1e-15)


@pytest.mark.parametrize("n,reps,gamma", [(6, 2, 0.5), (5, 3, 1.3), (4, 1, 0.1)])
def test_statevector_closed_form_d0(n, reps, gamma):
    rng = np.random.default_rng(n)
    X = rng.uniform(-2, 2, size=(5, n))
    K = statevector.gram(X, 0, reps, gamma)
    for i in range(5):
        for j in range(5):
            assert K[i, j] == pytest.approx(overlap.product_state_kernel(X[i], X[j], reps, gamma), abs=1e-14)


def test_statevector_invariants():
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(12, 7))
    K = statevector.gram(X, 3, 2, 0.8)
    assert np.allclose(np.diag(K), 1.0, atol=1e-13)
    assert np.allclose(K, K.T, atol=1e-15)
    assert K.min() >= 0 and K.max() <= 1 + 1e-13
    assert np.linalg.eigvalsh(K).min() > -1e-12      # Schur product of two PSD Gram matrices


def test_features_equal_one_switch_off_xx():
    """x_k = 1 for every feature makes every Rxx angle zero: product-state kernel."""
    n = 6
    a = np.ones(n)
    b = np.ones(n)
    b[2] = 0.999999  # still nearly one: its terms stay tiny but nonzero
    K = statevector.gram(np.stack([a, np.ones(n)]), 4, 2, 0.7)
    assert K[0, 1] == pytest.approx(1.0, abs=1e-14)
    c = np.linspace(-1, 1, n)
    # pairs with one all-ones vector still see Rxx on the other state, so only check a vs a
    sv = statevector.state(a, 5, 3, 0.7)
    prod = statevector.state(a, 0, 3, 0.7)
    assert np.allclose(sv, prod, atol=1e-15)


@pytest.mark.parametrize("n,d,reps,gamma", [(6, 1, 2, 0.5), (8, 1, 2, 0.5), (7, 3, 2, 0.9),
                                              (9, 4, 1, 1.3), (10, 2, 3, 0.6), (6, 5, 2, 0.8)])
def test_exact_mps_matches_statevector(n, d, reps, gamma):
    rng = np.random.default_rng(100 + n * 10 + d)
    for _ in range(3):
        x = rng.uniform(-1.5, 1.5, n)
        r = mps.build_mps(x, d, reps, gamma, chi_max=1 << 20, eps=0.0)
        v = mps.to_statevector(r.sites)
        ref = statevector.state(x, d, reps, gamma)
        assert np.max(np.abs(v - ref)) < 1e-13
        # exact bond dimensions never exceed the Schmidt bound
        for k in range(n + 1):
            assert r.bond_dims[k] <= min(2 ** k, 2 ** (n - k))


def test_left_canonical_and_normalised():
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, 14)
    r = mps.build_mps(x, 3, 2, 0.7, chi_max=12, eps=1e-6)
    for k, A in enumerate(r.sites[:-1]):
        M = A.reshape(-1, A.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(A.shape[2]), atol=1e-13)
    assert np.linalg.norm(r.sites[-1]) == pytest.approx(1.0, abs=1e-13)
    assert overlap.kernel_entry(r.sites, r.sites) == pytest.approx(1.0, abs=1e-13)


def test_d0_mps_is_product_state():
    rng = np.random.default_rng(3)
    X = rng.uniform(-2, 2, size=(4, 40))
    S = [mps.build_mps(x, 0, 2, 0.3, chi_max=8, eps=1e-8) for x in X]
    for r in S:
        assert list(r.bond_dims) == [1] * 41
    for i in range(4):
        for j in range(4):
            want = overlap.product_state_kernel(X[i], X[j], 2, 0.3)
            assert overlap.kernel_entry(S[i].sites, S[j].sites) == pytest.approx(want, rel=1e-12, abs=1e-300)


def test_truncation_bound_eq8():
    """Eq. 8: one cut at discarded weight w leaves fidelity 1 - w; over many
    cuts the infidelity with the exact state stays within the summed weights."""
    rng = np.random.default_rng(11)
    for trial in range(3):
        x = rng.uniform(-1.5, 1.5, 12)
        exact = statevector.state(x, 4, 2, 1.1)
        for eps, chi in ((1e-3, 64), (1e-2, 64), (0.0, 6)):
            r = mps.build_mps(x, 4, 2, 1.1, chi_max=chi, eps=eps)
            v = mps.to_statevector(r.sites)
            infid = 1.0 - abs(np.vdot(exact, v)) ** 2
            assert r.trunc_weight > 0
            assert infid <= 2.0 * r.trunc_weight + 1e-13
            assert infid >= -1e-13


def test_truncation_rank_rule():
    s = np.array([0.9, 0.4, 1e-3, 1e-8, 1e-9])
    s = s / np.linalg.norm(s)
    tot = 1.0
    # eps^2 = 1e-12: drop values whose squared tail <= 1e-12
    r, w, m, cap, gap = mps.truncation_rank(s, 10, 1e-6)
    assert r == 3 and not cap
    assert w == pytest.approx((s[3] ** 2 + s[4] ** 2), rel=1e-12)
    r, *_ = mps.truncation_rank(s, 10, 1e-1)  # tail after 2 values is 1e-6 <= 1e-2
    assert r == 2
    r, _, _, cap, gap = mps.truncation_rank(s, 1, 1e-9)
    assert r == 1 and cap
    r, *_ = mps.truncation_rank(s, 10, 0.0)
    assert r == 5
    # never below one value, even if everything could go
    r, *_ = mps.truncation_rank(np.array([1.0, 0.0]), 10, 0.5)
    assert r == 1


@pytest.mark.parametrize("n,d", [(8, 2), (11, 3)])
def test_overlap_matches_statevector(n, d):
    rng = np.random.default_rng(n)
    X = rng.uniform(-1, 1, size=(5, n))
    S = [mps.build_mps(x, d, 2, 0.8, chi_max=1 << 20, eps=0.0).sites for x in X]
    SV = np.stack([statevector.state(x, d, 2, 0.8) for x in X])
    for i in range(5):
        for j in range(5):
            z = overlap.sweep_left_to_right(S[i], S[j])
            assert abs(z - np.vdot(SV[i], SV[j])) < 1e-13
            assert abs(z - overlap.sweep_right_to_left(S[i], S[j])) < 1e-13


def test_tiny_workload_gram_vs_statevector():
    """n=8, d=1, r=2, gamma=0.5, 64 vectors: the full Gram against the
    256-amplitude statevector kernel."""
    import workloads
    w = workloads.tiny()
    S = [mps.build_mps(x, w.d, w.reps, w.gamma, w.chi_max, w.eps).sites for x in w.X]
    K = overlap.gram(S)
    Kref = statevector.gram(w.X, w.d, w.reps, w.gamma)
    assert np.max(np.abs(K - Kref)) < 1e-13
