"""GPU parity of qk_build_states against the CPU oracle (FP64 builder)."""
import numpy as np
import pytest

import workloads
from oracle import mps, overlap, statevector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import torch
    assert torch.cuda.is_available()
    import paper_2411_09336_gb300 as qk
    return qk


def rank_mismatches(ref_results, trace, reps_ops):
    """Rank decisions that differ from the oracle, minus the excused near-ties
    (tail sum within 1e-6 of its threshold, or a chi_max cut between two
    singular values closer than 1e-10 relative)."""
    bad = []
    for s, r in enumerate(ref_results):
        for o in range(reps_ops):
            if trace[s, o] != r.ranks[o]:
                if r.margins[o] < 1e-6 or (r.capped[o] and r.cap_gaps[o] < 1e-10):
                    continue
                bad.append((s, o, int(trace[s, o]), int(r.ranks[o])))
                break  # later ops of this state are downstream of the mismatch
    return bad


def test_tiny_exact_states_match_statevector(qk):
    w = workloads.tiny()
    A = qk.qk_build_states(w.X, w.d, w.reps, w.gamma, w.chi_max, w.eps, store="c128")
    dims = A.bond_dims()
    assert dims.shape == (64, 9)
    for s in range(0, 64, 7):
        ref = mps.build_mps(w.X[s], w.d, w.reps, w.gamma, w.chi_max, w.eps)
        assert list(dims[s]) == list(ref.bond_dims)
        v = mps.to_statevector(A.export(s))
        sv = statevector.state(w.X[s], w.d, w.reps, w.gamma)
        assert np.max(np.abs(v - sv)) < 1e-13
    K, _ = qk.qk_gram(A, prec="fp64")
    Kref = statevector.gram(w.X, w.d, w.reps, w.gamma)
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < 1e-12
    # the stored statevector Gram (tests/golden), FP64 and split paths
    from test_golden import load_tiny_golden
    Kg = load_tiny_golden()
    assert np.max(np.abs(K.cpu().numpy() - Kg)) < 1e-12
    Ks, _ = qk.qk_gram(A, prec="split")
    assert np.max(np.abs(Ks.cpu().numpy() - Kg)) < 1e-5


@pytest.mark.parametrize("n,d,reps,gamma,chi,eps,N", [
    (12, 3, 2, 0.9, 64, 0.0, 5),      # exact, wider blocks
    (10, 9, 1, 1.1, 64, 0.0, 3),      # d = n-1
    (9, 2, 3, 0.7, 64, 1e-8, 7),      # truncation on
])
def test_small_states_match_statevector(qk, n, d, reps, gamma, chi, eps, N):
    X = workloads.random_rows(n, N, seed=n * 100 + d)
    A = qk.qk_build_states(X, d, reps, gamma, chi, eps, store="c128")
    K, _ = qk.qk_gram(A, prec="fp64")
    Kref = statevector.gram(X, d, reps, gamma)
    tol = 1e-12 if eps == 0 else 1e-7
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < tol
    for s in range(N):
        assert abs(np.vdot(mps.to_statevector(A.export(s)), statevector.state(X[s], d, reps, gamma))) ** 2 \
            == pytest.approx(1.0, abs=1e-12 if eps == 0 else 1e-8)


def test_c50_ranks_and_kernel(qk):
    import torch
    w = workloads.c50(N=12)
    nops = qk.qk_schedule_length(w.n, w.d) * w.reps
    trace = torch.zeros((12, nops), dtype=torch.int32, device="cuda")
    A = qk.qk_build_states(w.X, w.d, w.reps, w.gamma, w.chi_max, w.eps, store="c128", rank_trace=trace)
    trace = trace.cpu().numpy()
    refs = [mps.build_mps(x, w.d, w.reps, w.gamma, w.chi_max, w.eps) for x in w.X]
    assert rank_mismatches(refs, trace, nops) == []
    dims = A.bond_dims()
    for s in range(12):
        assert list(dims[s]) == list(refs[s].bond_dims)
        assert A.trunc_weight()[s] == pytest.approx(refs[s].trunc_weight, rel=1e-3, abs=1e-20)
    K, _ = qk.qk_gram(A, prec="fp64")
    Kref = overlap.gram([r.sites for r in refs])
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < 1e-12


@pytest.mark.parametrize("name,count", [("c100", 3), ("c165", 2)])
def test_full_size_workloads_sampled(qk, name, count):
    """Full-size circuits (n=100 d=4, n=165 d=6, chi_max 128), a few states
    each: ranks, bond dims and kernel entries against the oracle."""
    import torch
    w = workloads.BY_NAME[name]()
    X = w.X[:count]
    nops = qk.qk_schedule_length(w.n, w.d) * w.reps
    trace = torch.zeros((count, nops), dtype=torch.int32, device="cuda")
    A = qk.qk_build_states(X, w.d, w.reps, w.gamma, w.chi_max, w.eps, store="c128", rank_trace=trace)
    refs = [mps.build_mps(x, w.d, w.reps, w.gamma, w.chi_max, w.eps) for x in X]
    assert rank_mismatches(refs, trace.cpu().numpy(), nops) == []
    K, _ = qk.qk_gram(A, prec="fp64")
    Kref = overlap.gram([r.sites for r in refs])
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < 1e-12
    assert np.allclose(np.diag(K.cpu().numpy()), 1.0, atol=1e-12)


def test_edge_cases(qk):
    # d = 0: product states, closed form
    X = workloads.random_rows(30, 4, seed=3)
    A = qk.qk_build_states(X, 0, 2, 0.4, 8, 1e-8)
    assert (A.bond_dims() == 1).all()
    K, _ = qk.qk_gram(A, prec="fp64")
    for i in range(4):
        for j in range(4):
            assert K[i, j].item() == pytest.approx(overlap.product_state_kernel(X[i], X[j], 2, 0.4),
                                                   rel=1e-6, abs=1e-30)
    # n = 2, N = 1
    X = workloads.random_rows(2, 1, seed=4)
    A = qk.qk_build_states(X, 1, 1, 0.8, 4, 0.0, store="c128")
    v = mps.to_statevector(A.export(0))
    assert np.allclose(v, statevector.state(X[0], 1, 1, 0.8), atol=1e-14)
    # chi_max = 1: every cut keeps one value; states stay normalised
    X = workloads.random_rows(10, 3, seed=5)
    A = qk.qk_build_states(X, 2, 2, 0.9, 1, 1e-8, store="c128")
    assert (A.bond_dims() == 1).all()
    K, _ = qk.qk_gram(A, prec="fp64")
    assert np.allclose(np.diag(K.cpu().numpy()), 1.0, atol=1e-12)
    refs = [mps.build_mps(x, 2, 2, 0.9, 1, 1e-8) for x in X]
    assert np.max(np.abs(K.cpu().numpy() - overlap.gram([r.sites for r in refs]))) < 1e-12
    # large eps: rank 1 everywhere
    A = qk.qk_build_states(X, 2, 2, 0.9, 16, 0.9, store="c128")
    assert (A.bond_dims() == 1).all()
    # invalid input is rejected with a clear error
    with pytest.raises(qk.QKError):
        qk.qk_build_states(np.full((2, 5), np.nan), 1, 1, 0.5, 4, 0.0)
