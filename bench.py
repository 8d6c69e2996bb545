#!/usr/bin/env python
"""Throughput benchmark: quantum-kernel Gram entries per second on GB300.

Workload (the n=165 circuit of the headline metric): n=165 qubits/features,
interaction distance d=6, r=2 repetitions, gamma=0.15, chi_max=128,
truncation eps=1e-8, complex64 states; synthetic stand-in for the Elliptic
data (standardised correlated Gaussian features, 6400 training rows).

Setup (untimed): each rank builds `--distinct` states from its own training
rows with the FP64 builder, then expands them to `--n-states` distinct
states by a final random Rz layer per copy (single-qubit Z rotations
contracted into the sites: bond profiles unchanged, overlaps between copies
as small as between different data points).

Step (timed): one qk_gram call on the resident batch - the symmetric Gram
(i <= j contracted and mirrored) by the split-precision tensor-core sweep,
with FP64 re-evaluation of the entries above 1e-3 (the diagonal).  value =
computed entries (N(N+1)/2 per rank, summed over ranks) / max-over-ranks time.
Inputs (the packed states, GBs) are far larger than L2.

--impl reference times the CPU oracle (numpy, FP64) on a bounded sample of
the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gram entries/s (n=165, chi=128), split-precision vs FP64 path on 1 GB300 at |dK|<=1e-5"

# DRAM bytes (read + write) per off-diagonal pair of tc_overlap_kernel<2> at
# the n=165, d=6, chi_max=128 circuit, from one ncu capture of a 192-state
# symmetric Gram (18,336 pairs, 568.2 GB in one launch).  The roofline's
# `traffic` scales it to the pairs of one launch; it holds only for that
# kernel version, the split depth P=2 and the tile schedule it was taken
# with (4 kets per tile, bands of 16 bras); another schedule reports null.
TC_DRAM_BYTES_PER_PAIR = 568.189336e9 / 18336
TC_TRAFFIC_SCHEDULE = {"kets_per_tile": 4, "band": 16}


def roofline_traffic(prec, schedule, pairs):
    """DRAM bytes of one tensor-core launch over `pairs` pairs, from the ncu
    per-pair figure; None unless the run used the captured depth and tile
    schedule."""
    if prec != "split" or not schedule:
        return None
    if any(schedule.get(k) != v for k, v in TC_TRAFFIC_SCHEDULE.items()):
        return None
    return TC_DRAM_BYTES_PER_PAIR * pairs


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-states", type=int, default=1824)
    p.add_argument("--distinct", type=int, default=152)
    p.add_argument("--prec", default="split", choices=["split", "split_bf16x3", "fp64"])
    p.add_argument("--fp64-sample", type=int, default=1, help="0 skips the FP64-path comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_rows(X: np.ndarray, rank: int, distinct: int) -> np.ndarray:
    """Training rows of one rank: disjoint consecutive blocks, so every rank
    builds and contracts its own independent batch (weak scaling)."""
    rows = X[rank * distinct:(rank + 1) * distinct]
    if len(rows) != distinct:
        raise ValueError(f"rank {rank}: only {len(rows)} of {distinct} training rows left")
    return rows


def max_over_ranks(ms: float, world: int, device: str = "cuda") -> float:
    """The step time every rank reports: the slowest rank's."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- helpers
def gram_flops(dims: np.ndarray, diagonal: bool = False) -> float:
    """Algorithmic real FLOPs of the pairs (bra i, ket j), i < j (and i = j
    when `diagonal`): per pair and site, T_s = E B[s] then
    E' = sum_s A[s]^H T_s, i.e. 2 (chi^a_k chi^b_k chi^b_k+1 +
    chi^a_k+1 chi^a_k chi^b_k+1) complex MACs, 8 real FLOPs each.  The count
    is not symmetric in (i, j), so it is summed in order with prefix sums."""
    c = dims.astype(np.float64)
    c0, c1 = c[:, :-1], c[:, 1:]
    bra1, ket1 = c0, c0 * c1          # chi^a_k      * (chi^b_k chi^b_k+1)
    bra2, ket2 = c1 * c0, c1          # chi^a_k+1 chi^a_k * chi^b_k+1
    pre1 = np.cumsum(bra1, axis=0) - bra1  # sum over i < j
    pre2 = np.cumsum(bra2, axis=0) - bra2
    total = np.sum(ket1 * pre1) + np.sum(ket2 * pre2)
    if diagonal:
        total += np.sum(bra1 * ket1 + bra2 * ket2)
    return 16.0 * total


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---- the CPU oracle on the host cores: one spawned process per core, each
# with one BLAS thread, each holding the same 3 oracle-built c165 states
_ORACLE_STATES = None
_ORACLE_PAIRS = [(i, j) for i in range(3) for j in range(i, 3)]
_ONE_THREAD = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def _oracle_init():
    global _ORACLE_STATES
    import workloads
    from oracle import mps
    w = workloads.c165()
    _ORACLE_STATES = [mps.build_mps(x, w.d, w.reps, w.gamma, w.chi_max, w.eps).sites for x in w.X_train[:3]]


def _oracle_round(_):
    from oracle import overlap
    for i, j in _ORACLE_PAIRS:
        overlap.kernel_entry(_ORACLE_STATES[i], _ORACLE_STATES[j])
    return len(_ORACLE_PAIRS)


def _oracle_for(seconds):
    done, t0 = 0, time.time()
    while time.time() - t0 < seconds:
        done += _oracle_round(0)
    return done, time.time() - t0


class OraclePool:
    """Spawned worker processes (safe after CUDA initialisation), BLAS
    threads pinned to one per process; the state build is not timed."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in _ONE_THREAD}
        os.environ.update(_ONE_THREAD)
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        t0 = time.time()
        self.pool.map(_oracle_round, range(self.procs), chunksize=1)  # waits for the builds
        self.build_s = time.time() - t0

    def round(self):
        """One pass over the 6 pairs in every process; entries computed."""
        return sum(self.pool.map(_oracle_round, range(self.procs), chunksize=1))

    def run_for(self, seconds):
        """Every process sweeps for `seconds`; returns (entries, summed
        per-process rate), each process timing its own loop."""
        res = self.pool.map(_oracle_for, [seconds] * self.procs, chunksize=1)
        return sum(n for n, _ in res), sum(n / dt for n, dt in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_rate(target_s: float = 15.0):
    """The CPU oracle (numpy FP64 transfer sweeps) on a bounded sample: every
    process repeats the 6 overlaps (i <= j) of 3 oracle-built c165 states for
    about target_s seconds."""
    op = OraclePool()
    try:
        done, rate = op.run_for(target_s)
    finally:
        op.close()
    return rate, {"entries": done, "seconds": round(target_s, 2), "procs": op.procs,
                  "build_s": round(op.build_s, 1)}


# --------------------------------------------------------------------- reference arm
def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    op = OraclePool()
    try:
        for _ in range(a.warmup):
            op.round()
        t0 = time.time()
        n = sum(op.round() for _ in range(a.steps))
        dt = time.time() - t0
    finally:
        op.close()
    v = n / dt
    sample = (f"{op.procs} processes x 6 numpy transfer-sweep overlaps (i <= j) of 3 oracle-built c165 "
              f"states per step, one BLAS thread each")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "entries/s", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * dt / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "c165: n=165 d=6 r=2 gamma=0.15 chi_max=128 eps=1e-8", "sample": sample},
           "cpu_baseline": {"value": v, "unit": "entries/s", "cores": op.procs, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2411_09336_gb300 as qk
    import workloads

    w = workloads.c165()
    rows = rank_rows(w.X_train, rank, a.distinct)
    stream = torch.cuda.current_stream()

    # ---- setup: FP64 builder, then rotated copies
    torch.cuda.synchronize()
    t0 = time.time()
    base = qk.qk_build_states(rows, w.d, w.reps, w.gamma, w.chi_max, w.eps, store="c64")
    torch.cuda.synchronize()
    build_s = time.time() - t0
    copies = max(1, a.n_states // a.distinct)
    rng = np.random.default_rng(1000 + rank)
    phi = rng.uniform(-math.pi, math.pi, size=(copies, w.n))
    phi[0] = 0.0  # copy 0 is the built states themselves
    A = qk.qk_mps_rz_copies(base, phi)
    N = A.N
    dims = A.bond_dims()
    flops = gram_flops(dims)

    def step():
        K, nref = qk.qk_gram(A, prec=a.prec, out=Kbuf)
        return nref

    Kbuf = torch.empty((N, N), dtype=torch.float64, device="cuda")
    for _ in range(a.warmup):
        step()  # the first split call also tunes the tile schedule
    schedule = qk.qk_tune_split(A, prec=a.prec) if a.prec != "fp64" else None
    # ---- timed region
    sampler = ClockSampler(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    kern_ms, refine_ms, nrefs = [], [], []
    for _ in range(a.steps):
        nrefs.append(step())
        prof = qk.qk_last_profile()
        kern_ms.append(prof["overlap_ms"])
        refine_ms.append(prof["refine_ms"])
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    entries = N * (N + 1) // 2
    value = entries * world * a.steps / (ms / 1000.0)

    # ---- FP64 path on the same GPU, on the built (distinct) states
    fp64 = None
    if a.prec != "fp64" and a.fp64_sample > 0:
        sub = base
        Ks, _ = qk.qk_gram(sub, prec=a.prec)
        torch.cuda.synchronize()
        t0 = time.time()
        K64, _ = qk.qk_gram(sub, prec="fp64")
        torch.cuda.synchronize()
        dt = time.time() - t0
        e64 = sub.N * (sub.N + 1) // 2
        fp64 = {"value": e64 / dt, "unit": "entries/s", "states": sub.N,
                "max_abs_dK_split_vs_fp64": float((Ks - K64).abs().max().item())}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        nb = qk.qk_mps_blob_bytes(A)
        blob = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        qk.qk_mps_save(A, blob)
        Kh = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.time()
        for _ in range(a.steps):
            # a fresh batch per step: the tile schedule tuned above is found
            # again by the Gram's shape, not re-timed
            B = qk.qk_mps_load(blob)
            qk.qk_gram(B, prec=a.prec, out=Kh)
            B.free()
        torch.cuda.synchronize()
        dt = max_over_ranks(1000.0 * (time.time() - t0), world) / 1000.0
        e2e = {"value": entries * world * a.steps / dt, "unit": "entries/s", "h2d_bytes_per_step": int(nb),
               "d2h_bytes_per_step": int(N * N * 8), "steps": a.steps}

    # kernels of one split qk_gram on a symmetric batch: the tensor-core sweep,
    # the self-overlaps, the refinement selection, and, when entries were
    # selected, the FP64 sweep over them and their scatter into K
    if a.prec == "fp64":
        launches = a.steps
    else:
        launches = sum(3 + (2 if r > N else 0) for r in nrefs)
    pairs = N * (N - 1) // 2
    traffic = roofline_traffic(a.prec, schedule, pairs)
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    kavg = float(np.mean(kern_ms)) if kern_ms else float("nan")
    achieved = flops / (kavg / 1000.0) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x2-split->f32" if a.prec == "split" else
        ("bf16x3-split->f32" if a.prec == "split_bf16x3" else "f64"),
        "data": "synthetic",
        "config": {"workload": "c165: n=165 d=6 r=2 gamma=0.15 chi_max=128 eps=1e-8, complex64 states",
                   "states_per_rank": N, "distinct_built_per_rank": a.distinct,
                   "expansion": f"{copies} copies per built state via a random final Rz layer",
                   "gram": "symmetric, i<=j contracted, FP64 re-evaluation above 1e-3",
                   "prec": a.prec, "l2": "inputs larger than L2 (packed states GBs)",
                   "mean_chi": float(dims.mean()), "max_chi": int(dims.max()),
                   "tile_schedule": schedule},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "tc_overlap_kernel", "peak_source": f"bf16_tflops_sustained ({src})",
                     "algorithmic_tflop_per_launch": flops / 1e12,
                     "kernel_ms_per_launch": kavg, "refine_ms_per_step": float(np.mean(refine_ms)),
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of a 192-state "
                                        "capture, per pair, times the launch's pairs") if traffic else
                                       ("null: the ncu capture was taken with the schedule "
                                        f"{TC_TRAFFIC_SCHEDULE}, this run used {schedule}"),
                     "dram_tb_per_s": (traffic / (kavg / 1000.0) / 1e12) if traffic else None,
                     "note": "algorithmic complex-MAC FLOPs; the bf16x2 split issues 3 bf16 products per "
                             "real product, so frac <= 1/3 at full tensor-pipe use"},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": e2e,
        "fp64_path": fp64,
        "builder": {"states": base.N, "seconds": round(build_s, 1), "states_per_s": base.N / build_s},
        "n_refined_per_step": int(np.mean(nrefs)) if nrefs else 0,
    }
    if rank == 0 and not a.no_cpu_baseline:
        v, sample = cpu_oracle_rate()
        out["cpu_baseline"] = {"value": v, "unit": "entries/s", "cores": sample["procs"], "kind": "oracle",
                               "sample": f"{sample['entries']} numpy transfer-sweep overlaps among 3 "
                                         f"oracle-built c165 states in {sample['seconds']} s on "
                                         f"{sample['procs']} processes with one BLAS thread each "
                                         f"(state build {sample['build_s']} s, excluded)"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
