"""GPU parity of the FP64 transfer sweep on identical (imported) states."""
import numpy as np
import pytest

import workloads
from oracle import mps, overlap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import paper_2411_09336_gb300 as qk
    return qk


@pytest.fixture(scope="module")
def states():
    # ragged bond dimensions: mixed d, truncation and chi caps, 23 states
    out = []
    rng = np.random.default_rng(9)
    for s in range(23):
        x = rng.uniform(-1.5, 1.5, 14)
        d = 1 + s % 4
        chi = [4, 9, 16, 33][s % 4]
        out.append(mps.build_mps(x, d, 2, 0.8, chi, 1e-10).sites)
    return out


@pytest.mark.parametrize("store", ["c128", "c64"])
def test_symmetric_gram(qk, states, store):
    A = qk.qk_mps_import(states, store=store)
    K, _ = qk.qk_gram(A, prec="fp64")
    ref_states = [mps.round_sites(s, store) for s in states]
    Kref = overlap.gram(ref_states)
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < 1e-12
    assert np.array_equal(K.cpu().numpy(), K.cpu().numpy().T)


def test_rectangular_and_pairs(qk, states):
    A = qk.qk_mps_import(states[:9], store="c128")
    B = qk.qk_mps_import(states[9:], store="c128")
    K, _ = qk.qk_gram(A, B, prec="fp64")
    Kref = overlap.gram(states[:9], states[9:])
    assert K.shape == (9, 14)
    assert np.max(np.abs(K.cpu().numpy() - Kref)) < 1e-12
    pairs = np.array([[0, 0], [8, 13], [3, 7], [3, 7], [5, 1]], dtype=np.int32)
    kp = qk.qk_gram_pairs(A, B, pairs, prec="fp64").cpu().numpy()
    assert np.allclose(kp, Kref[pairs[:, 0], pairs[:, 1]], rtol=0, atol=1e-12)
    # host output buffer
    out = np.zeros((9, 14))
    qk.qk_gram(A, B, prec="fp64", out=out)
    assert np.max(np.abs(out - Kref)) < 1e-12
    # out-of-range pair index is rejected
    with pytest.raises(qk.QKError):
        qk.qk_gram_pairs(A, B, np.array([[9, 0]], dtype=np.int32), prec="fp64")


def test_roundtrip_export(qk, states):
    A = qk.qk_mps_import(states[:4], store="c128")
    for s in range(4):
        got = A.export(s)
        for g, r in zip(got, states[s]):
            assert np.array_equal(g, r)
