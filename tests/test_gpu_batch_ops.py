"""GPU checks of the batch utilities: rotated copies against the oracle's
Z layer, and the host-blob save/load round trip."""
import numpy as np
import pytest

from oracle import mps, overlap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import paper_2411_09336_gb300 as qk
    return qk


def test_rz_copies_match_oracle_z_layer(qk):
    rng = np.random.default_rng(2)
    n = 9
    st = [mps.build_mps(rng.uniform(-1, 1, n), 2, 2, 0.7, 16, 1e-10).sites for _ in range(3)]
    A = qk.qk_mps_import(st, store="c128")
    phi = rng.uniform(-np.pi, np.pi, size=(2, n))
    B = qk.qk_mps_rz_copies(A, phi)
    assert B.N == 6
    assert np.array_equal(B.bond_dims()[:3], A.bond_dims())
    ref = []
    for c in range(2):
        for s in range(3):
            sites = [x.copy() for x in st[s]]
            # the Z layer of Eq. 4 with phases phi: slice q times exp(-i phi (1 - 2q))
            for k in range(n):
                sites[k] = sites[k] * np.array([np.exp(-1j * phi[c, k]), np.exp(1j * phi[c, k])]).reshape(1, 2, 1)
            ref.append(sites)
    K, _ = qk.qk_gram(B, prec="fp64")
    assert np.max(np.abs(K.cpu().numpy() - overlap.gram(ref))) < 1e-12


def test_save_load_roundtrip(qk):
    import torch
    rng = np.random.default_rng(3)
    st = [mps.build_mps(rng.uniform(-1, 1, 11), 3, 2, 0.9, 20, 1e-9).sites for _ in range(4)]
    A = qk.qk_mps_import(st, store="c64")
    nb = qk.qk_mps_blob_bytes(A)
    for blob in (np.zeros(nb, dtype=np.uint8), torch.zeros(nb, dtype=torch.uint8, device="cuda")):
        qk.qk_mps_save(A, blob)
        B = qk.qk_mps_load(blob)
        assert np.array_equal(B.bond_dims(), A.bond_dims())
        for s in range(4):
            for x, y in zip(A.export(s), B.export(s)):
                assert np.array_equal(x, y)
    bad = np.zeros(64, dtype=np.uint8)
    with pytest.raises(qk.QKError):
        qk.qk_mps_load(bad)
