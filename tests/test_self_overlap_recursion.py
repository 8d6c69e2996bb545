"""The self-overlap recursion used by the split path for K_ii, as algebra on
the CPU: for a left-canonical MPS the transfer sweep of a state with itself
keeps E = I + F small-F, with F_{k+1} = G_k + sum_s A_k[s]^H F_k A_k[s] and
G_k = sum_s A_k[s]^H A_k[s] - I.  Forming G in FP64 and running F in
complex64 must reproduce the oracle's FP64 transfer sweep (Fig. 2) to
~1e-12; states that are not left-canonical show a defect far above the
1e-4 limit at which the GPU path falls back to the FP64 sweep.  (The GPU
kernel itself is checked against the FP64 sweep in the gpu tests.)"""
import numpy as np
import pytest

from oracle import mps, overlap


def defect(a):
    """G = sum_s A[s]^H A[s] - I for a site a[chi_l, s, chi_r], in FP64."""
    a = a.astype(np.complex128)
    return np.einsum("xsu,xsv->uv", a.conj(), a) - np.eye(a.shape[2])


def self_overlap_by_recursion(sites):
    F = np.zeros((1, 1), np.complex64)
    for a in sites:
        a32 = a.astype(np.complex64)
        T = np.einsum("xc,csv->xsv", F, a32)
        F = (defect(a).astype(np.complex64) + np.einsum("xsu,xsv->uv", a32.conj(), T)).astype(np.complex64)
    z = 1.0 + complex(F[0, 0])
    return abs(z) ** 2


def states(count, n=12, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        x = rng.uniform(-1.5, 1.5, n)
        r = mps.build_mps(x, 1 + s % 3, 2, 0.9, (8, 16, 32)[s % 3], 1e-10)
        out.append(mps.round_sites(r.sites, "c64"))
    return out


def test_recursion_matches_fp64_sweep():
    for st in states(6):
        ref = overlap.kernel_entry(st, st)
        assert max(np.abs(defect(a)).max() for a in st) < 1e-6      # complex64 rounding only
        assert abs(self_overlap_by_recursion(st) - ref) <= 1e-12


def test_recursion_with_norm_defect_on_last_site():
    for st in states(3, seed=8):
        st = [a.copy() for a in st]
        st[-1] = (st[-1] * (1 + 3e-6)).astype(np.complex64)
        ref = overlap.kernel_entry(st, st)
        assert abs(ref - 1.0) > 1e-5                                  # the defect shows in K_ii
        assert abs(self_overlap_by_recursion(st) - ref) <= 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_not_left_canonical_is_detected(seed):
    rng = np.random.default_rng(seed)
    chis = [1, 2, 4, 4, 2, 1]
    st = [(rng.standard_normal((chis[k], 2, chis[k + 1])) + 1j * rng.standard_normal((chis[k], 2, chis[k + 1])))
          / (2 * np.sqrt(chis[k])) for k in range(5)]
    assert max(np.abs(defect(a)).max() for a in st) > 1e-4
    # a right-canonical form of a left-canonical state is not left-canonical
    st = states(1)[0]
    flipped = [np.transpose(a, (2, 1, 0)).conj() for a in reversed(st)]
    assert max(np.abs(defect(a)).max() for a in flipped) > 1e-4
