"""Host-side logic of bench.py: the algorithmic FLOP count against brute
force, and the multi-rank sharding / max-over-ranks timing on two gloo
ranks (CPU)."""
import os
import socket

import numpy as np
import pytest

import bench


def test_gram_flops_brute_force():
    rng = np.random.default_rng(0)
    N, n = 7, 9
    dims = np.ones((N, n + 1), dtype=np.int64)
    dims[:, 1:-1] = rng.integers(1, 40, size=(N, n - 1))
    strict, diag = 0.0, 0.0
    for i in range(N):
        for j in range(i, N):
            a, b = dims[i], dims[j]   # bra i, ket j
            f = sum(16.0 * (a[k] * b[k] * b[k + 1] + a[k + 1] * a[k] * b[k + 1]) for k in range(n))
            if i == j:
                diag += f
            else:
                strict += f
    assert bench.gram_flops(dims) == pytest.approx(strict, rel=1e-12)
    assert bench.gram_flops(dims, diagonal=True) == pytest.approx(strict + diag, rel=1e-12)


def test_gram_flops_min_order_brute_force():
    """The algorithmic count takes, per pair and site, the cheaper of the two
    contraction orders (E B first, or A^H E first)."""
    rng = np.random.default_rng(1)
    N, n = 6, 8
    dims = np.ones((N, n + 1), dtype=np.int64)
    dims[:, 1:-1] = rng.integers(1, 50, size=(N, n - 1))
    strict = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            a, b = dims[i], dims[j]
            for k in range(n):
                ca = a[k] * b[k] * b[k + 1] + a[k + 1] * a[k] * b[k + 1]
                cb = a[k + 1] * a[k] * b[k] + a[k + 1] * b[k] * b[k + 1]
                strict += 16.0 * min(ca, cb)
    got = bench.gram_flops(dims, order="min")
    assert got == pytest.approx(strict, rel=1e-12)
    assert got <= bench.gram_flops(dims)


def test_fp64_peak_from_unit_count():
    # 2 DFMA per clock per SM at 152 SMs and 2070 MHz: the nominal 1.25 TFLOP/s
    assert bench.fp64_peak_tflops(2070.0, 152) == pytest.approx(1.2586, rel=1e-3)


def test_rank_rows_disjoint_and_checked():
    X = np.arange(40 * 3, dtype=float).reshape(40, 3)
    blocks = [bench.rank_rows(X, r, 8) for r in range(5)]
    flat = np.concatenate([b[:, 0] for b in blocks])
    assert len(np.unique(flat)) == 40
    with pytest.raises(ValueError):
        bench.rank_rows(X, 5, 8)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = np.arange(100 * 2, dtype=float).reshape(100, 2)
    rows = bench.rank_rows(X, rank, 10)
    ms = bench.max_over_ranks([3.5, 7.25][rank], world, device="cpu")
    out.put((rank, ms, rows[:, 0].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == 7.25
    assert set(res[0][2]).isdisjoint(res[1][2])


def test_roofline_traffic_only_for_the_captured_schedule(monkeypatch):
    sch = dict(bench.BENCH_SCHEDULE)
    monkeypatch.setattr(bench, "TC_DRAM_BYTES_PER_PAIR", 1.5e6)
    assert bench.roofline_traffic("split", sch, 10) == 1.5e7
    assert bench.roofline_traffic("split", {**sch, "kets_per_tile": 4}, 10) is None
    assert bench.roofline_traffic("split_bf16x3", sch, 10) is None
    assert bench.roofline_traffic("fp64", None, 10) is None
    assert bench.roofline_traffic("split", {**sch, "us_per_pair": 7.0}, 10) is not None
    monkeypatch.setattr(bench, "TC_DRAM_BYTES_PER_PAIR", None)
    assert bench.roofline_traffic("split", sch, 10) is None


def test_issued_macs_follow_the_kernel_tiling():
    """Brute-force replay of the kernel's tile loops (one ket per tile)."""
    rng = np.random.default_rng(4)
    N, n = 5, 7
    dims = np.ones((N, n + 1), dtype=np.int64)
    dims[:, 1:-1] = rng.integers(1, 129, size=(N, n - 1))
    pad = lambda x: (int(x) + 15) // 16 * 16
    ref = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            for k in range(n):
                ap, ap1 = pad(dims[i, k]), pad(dims[i, k + 1])
                bp, bp1 = pad(dims[j, k]), pad(dims[j, k + 1])
                rows = 2 * bp1
                M, nt = (64, 1) if rows <= 64 else (128, (rows + 127) // 128)
                for _t in range(nt):
                    for h0 in range(0, ap, 64):
                        nh = min(64, ap - h0)
                        ref += (bp // 16) * 3 * 2 * M * (2 * nh) * 16      # HS1 chunks x MMAs
                M2 = 64 if ap1 <= 64 else 128
                for h0 in range(0, bp1, 64):
                    nh = min(64, bp1 - h0)
                    ref += (2 * ap // 16) * 3 * 2 * M2 * (2 * nh) * 16       # HS2
    assert bench.issued_macs(dims) == pytest.approx(ref, rel=1e-12)


def test_table3_data_scaled_into_0_2():
    import workloads
    w = workloads.c165()
    Xtr, ytr, Xte, yte = bench.table3_data(w, 1, 800, 200)
    assert Xtr.shape == (800, 50) and Xte.shape == (200, 50)
    assert np.allclose(Xtr.min(axis=0), 0.0) and np.allclose(Xtr.max(axis=0), 2.0)
    assert Xte.min() >= 0.0 and Xte.max() <= 2.0
    # rank 1 takes training rows 800..1599 and test rows 200..399
    raw = w.X_train[800:1600, :50]
    assert np.allclose(Xtr[:, 3], 2 * (raw[:, 3] - raw[:, 3].min()) / np.ptp(raw[:, 3]))
    assert np.array_equal(ytr, w.y[800:1600]) and np.array_equal(yte, w.y[6400 + 200:6400 + 400])
    with pytest.raises(ValueError):
        bench.table3_data(w, 8, 800, 200)
