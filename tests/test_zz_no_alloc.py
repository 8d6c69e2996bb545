"""GPU test of qk_gram_pairs_noalloc, the FP64 pair-overlap entry point that
allocates nothing (for callers that must not allocate during the work, e.g.
a host that owns the device memory pool).  It must agree with qk_gram_pairs
(FP64) within the FP64 path's tolerance on two calls in a row, which share
the static scratch.  Collected last on purpose (file name)."""
import numpy as np
import pytest

from oracle import mps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import paper_2411_09336_gb300 as qk
    return qk


def states(count, n, seed, chis):
    rng = np.random.default_rng(seed)
    return [mps.build_mps(rng.uniform(-1.5, 1.5, n), 1 + s % 4, 2, 0.8, chis[s % len(chis)], 1e-10).sites
            for s in range(count)]


def test_noalloc_matches_gram_pairs_twice(qk):
    import torch
    st = states(19, 13, 21, (4, 9, 16, 40, 64))
    A = qk.qk_mps_import(st[:8], store="c64")
    B = qk.qk_mps_import(st[8:], store="c64")
    rng = np.random.default_rng(3)
    pairs = np.stack([rng.integers(0, 8, 300), rng.integers(0, 11, 300)], axis=1).astype(np.int32)
    ref = qk.qk_gram_pairs(A, B, pairs, prec="fp64").cpu().numpy()
    dp = torch.from_numpy(pairs).cuda()
    for call in range(2):
        out = torch.full((len(pairs),), float("nan"), dtype=torch.float64, device="cuda")
        qk.qk_gram_pairs_noalloc(A, B, dp, out)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.max(np.abs(got - ref)) < 1e-12, call
    # a different, shorter pair list right after reuses the same scratch
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    qk.qk_gram_pairs_noalloc(A, B, dp[:5].contiguous(), out)
    assert np.max(np.abs(out.cpu().numpy() - ref[:5])) < 1e-12


def test_noalloc_rejects_what_it_cannot_hold(qk):
    import torch
    rng = np.random.default_rng(5)
    big = [mps.build_mps(rng.uniform(-1, 1, 16), 8, 2, 1.0, 128, 0.0).sites for _ in range(2)]
    assert max(a.shape[2] for s in big for a in s) > 64
    A = qk.qk_mps_import(big, store="c64")
    dp = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(qk.QKError, match="64"):
        qk.qk_gram_pairs_noalloc(A, A, dp, out)
    small = qk.qk_mps_import(states(3, 10, 6, (8,)), store="c64")
    with pytest.raises(qk.QKError):
        qk.qk_gram_pairs_noalloc(small, small, torch.tensor([[0, 3]], dtype=torch.int32, device="cuda"), out)
    with pytest.raises(ValueError):  # host output buffer
        qk.qk_gram_pairs_noalloc(small, small, dp, torch.empty(1, dtype=torch.float64))
    two = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):  # output shorter than the pair list
        qk.qk_gram_pairs_noalloc(small, small, two, out)
    with pytest.raises(ValueError):  # float32 output
        qk.qk_gram_pairs_noalloc(small, small, dp, torch.empty(1, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):  # int64 pairs
        qk.qk_gram_pairs_noalloc(small, small, dp.to(torch.int64), out)
    with pytest.raises(ValueError):  # pairs not of shape (P, 2)
        qk.qk_gram_pairs_noalloc(small, small, torch.zeros(2, dtype=torch.int32, device="cuda"), out)


def test_noalloc_allocates_no_device_memory(qk):
    """After a first call on the device, further calls leave the device's
    free memory and torch's caching allocator untouched."""
    import torch
    st = states(6, 11, 8, (8, 16))
    A = qk.qk_mps_import(st, store="c64")
    pairs = torch.tensor([[i, j] for i in range(6) for j in range(6)], dtype=torch.int32, device="cuda")
    out = torch.empty(len(pairs), dtype=torch.float64, device="cuda")
    qk.qk_gram_pairs_noalloc(A, A, pairs, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    qk.qk_gram_pairs_noalloc(A, A, pairs, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocated_bytes.all.current", "reserved_bytes.all.current", "allocation.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
