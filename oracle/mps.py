"""MPS simulation of the feature-map circuit with per-gate SVD truncation.

Follows Sec. II-B: site tensors A_k[a, s, b] (left bond, qubit, right bond;
Eq. 6/7 reshapes), single-qubit gates contracted into their site (Fig. 1a),
two-qubit gates contracted with both sites, split by SVD and the singular
values absorbed into one side (Fig. 1b).  Truncation (Eq. 8 and the text
after it): drop the smallest singular values while their squared sum stays
at or below eps^2 of the total, i.e. the discarded weight is <= eps^2
(eps = 1e-8 gives the paper's 1e-16).

Readings (the paper is silent on these):
  * Rank rule: r = min{ r >= 1 : sum_{i >= r} s_i^2 <= eps^2 * sum_i s_i^2 }
    (0-based, tail summed from the smallest value upward), then
    r = min(r, chi_max).  eps = 0 means no truncation below chi_max.
  * The kept singular values are rescaled to unit norm after every cut, so
    the state stays normalised (<psi|psi> = 1, hence K_ii = 1).
  * Canonical form (footnote of Sec. II-B): the orthogonality centre is kept
    on the two sites of every gate.  After an op at (p, p+1) the singular
    values go right (site p+1) when the next op lies to the right, else left
    (site p).  Between repetitions the centre walks back to the chain start
    by LQ steps; at the end it walks to the last site by QR steps, so the
    stored state is left-canonical.  QR/LQ use the reduced factorisation
    (new bond = min of the two sides).
  * Each scheduled op (circuit.schedule) is one 2-site gate and one SVD.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import circuit


@dataclass
class MPSResult:
    sites: list                  # A_k, shape (chi_k, 2, chi_{k+1}), complex128
    bond_dims: np.ndarray        # (n+1,) int, chi_0 = chi_n = 1
    trunc_weight: float          # sum over ops of discarded weight (pre-renormalisation)
    ranks: np.ndarray            # rank kept after every 2-site op, in execution order
    margins: np.ndarray          # relative distance of the rank decision from its threshold
    capped: np.ndarray           # bool per op: rank set by chi_max
    cap_gaps: np.ndarray         # relative gap s_{r-1} vs s_r where capped (else inf)
    spectra: list = field(default_factory=list)  # optional per-op singular values


def truncation_rank(s: np.ndarray, chi_max: int, eps: float):
    """Rank rule of Eq. 8 as read above.  Returns (r, discarded, margin, capped, gap)."""
    L = len(s)
    s2 = s * s
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[i] = sum_{j>=i} s2[j]
    tot = tail[0]
    margin = np.inf
    if eps > 0.0:
        thr = eps * eps * tot
        r = L
        for cand in range(1, L + 1):
            if tail[cand] <= thr:
                r = cand
                break
        if thr > 0.0:
            margin = abs(tail[r] - thr) / thr
            if r >= 2:
                margin = min(margin, abs(tail[r - 1] - thr) / thr)
    else:
        r = L
    capped = r > chi_max
    gap = np.inf
    if capped:
        r = chi_max
        gap = (s[r - 1] - s[r]) / s[r - 1] if s[r - 1] > 0 else 0.0
    return r, tail[r] / tot if tot > 0 else 0.0, margin, capped, gap


def _move_right(A, c):
    """QR step: centre from site c to c+1."""
    cl, _, cr = A[c].shape
    Q, R = np.linalg.qr(A[c].reshape(cl * 2, cr), mode="reduced")
    k = Q.shape[1]
    A[c] = Q.reshape(cl, 2, k)
    A[c + 1] = np.tensordot(R, A[c + 1], axes=(1, 0))


def _move_left(A, c):
    """LQ step: centre from site c to c-1."""
    cl, _, cr = A[c].shape
    Q, R = np.linalg.qr(A[c].reshape(cl, 2 * cr).conj().T, mode="reduced")
    k = Q.shape[1]
    A[c] = Q.conj().T.reshape(k, 2, cr)
    A[c - 1] = np.tensordot(A[c - 1], R.conj().T, axes=(2, 0))


def initial_sites(n: int):
    """|+>^n as n sites of shape (1, 2, 1) (Hadamard layer, Eq. 2)."""
    return [np.full((1, 2, 1), 1.0 / np.sqrt(2.0), dtype=np.complex128) for _ in range(n)]


def apply_z_layer(A, x, gamma):
    """exp(-i H_Z): site k slice s is scaled by exp(-i phi_k (1 - 2 s)) (Eq. 4, Fig. 1a)."""
    phi = circuit.z_phases(x, gamma)
    for k in range(len(A)):
        A[k] = A[k] * np.array([np.exp(-1j * phi[k]), np.exp(1j * phi[k])]).reshape(1, 2, 1)


def build_mps(x, d: int, reps: int, gamma: float, chi_max: int, eps: float,
              keep_spectra: bool = False) -> MPSResult:
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    A = initial_sites(n)
    ops = circuit.schedule(n, d)
    seq = [op for _ in range(reps) for op in ops]
    ranks, margins, capped, gaps, spectra = [], [], [], [], []
    wsum = 0.0
    centre = 0
    oi = 0
    for rep in range(reps):
        apply_z_layer(A, x, gamma)
        for op in ops:
            p = op.p
            # bring the orthogonality centre onto (p, p+1)
            while centre < p:
                _move_right(A, centre)
                centre += 1
            while centre > p + 1:
                _move_left(A, centre)
                centre -= 1
            cl = A[p].shape[0]
            cr = A[p + 1].shape[2]
            theta = np.tensordot(A[p], A[p + 1], axes=(2, 0)).reshape(cl, 4, cr)
            G = circuit.op_matrix(op, x, gamma)
            theta = np.einsum("gh,ahb->agb", G, theta).reshape(cl * 2, 2 * cr)
            U, s, Vh = np.linalg.svd(theta, full_matrices=False)
            r, w, m, cap, gap = truncation_rank(s, chi_max, eps)
            wsum += w
            ranks.append(r)
            margins.append(m)
            capped.append(cap)
            gaps.append(gap)
            if keep_spectra:
                spectra.append(s.copy())
            sk = s[:r] / np.sqrt(np.sum(s[:r] ** 2))
            nxt = seq[oi + 1].p if oi + 1 < len(seq) else n  # beyond the end: go right
            if nxt > p:
                A[p] = U[:, :r].reshape(cl, 2, r)
                A[p + 1] = (sk[:, None] * Vh[:r]).reshape(r, 2, cr)
                centre = p + 1
            else:
                A[p] = (U[:, :r] * sk[None, :]).reshape(cl, 2, r)
                A[p + 1] = Vh[:r].reshape(r, 2, cr)
                centre = p
            oi += 1
    while centre < n - 1:
        _move_right(A, centre)
        centre += 1
    dims = np.array([1] + [A[k].shape[2] for k in range(n - 1)] + [1], dtype=np.int64)
    return MPSResult(A, dims, wsum, np.array(ranks, dtype=np.int64), np.array(margins),
                     np.array(capped, dtype=bool), np.array(gaps), spectra)


def to_statevector(sites) -> np.ndarray:
    """Contract an MPS into its 2^n amplitudes (qubit 0 most significant)."""
    v = sites[0].reshape(2, -1)
    for A in sites[1:]:
        v = np.tensordot(v, A, axes=(1, 0)).reshape(-1, A.shape[2])
    return v.reshape(-1)


def round_sites(sites, store: str):
    """Storage rounding of a built state: 'c128' keeps FP64, 'c64' rounds re/im to FP32."""
    if store == "c128":
        return [A.copy() for A in sites]
    if store == "c64":
        return [A.astype(np.complex64).astype(np.complex128) for A in sites]
    raise ValueError(store)
