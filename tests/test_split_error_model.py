"""The error model behind the split path's parity bar (2e-3 relative on K
for entries above 1e-8, 1e-5 absolute), checked on the CPU.

The tensor-core sweep (Fig. 2) forms every half-step product from operands
split into bf16 parts, x = x_hi + x_lo with x_hi = bf16(x) and
x_lo = bf16(x - x_hi), keeps the products hi*hi, hi*lo and lo*hi, and
accumulates in FP32; the half-step result is rounded to FP32 and split again
for the next product.  This test restates that arithmetic in numpy (bf16
rounding to nearest even, each half-step's result rounded to FP32; the
order of the FP32 additions inside one MMA is not modelled) on oracle-built
states and compares |<a|b>|^2 with the FP64 sweep.  The relative error grows
like a random walk over the sites, about 2^-16 per operand rounding, so over
n = 60 sites it stays far inside the bar; dropping a cross term (a
plausible mistake) makes it fail."""
import numpy as np

from oracle import mps, overlap


def bf16(x):
    """Round float64 values to bf16 (nearest even) through FP32."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def split(x):
    hi = bf16(x)
    return hi, bf16(x - hi)


def cmat_split(M):
    (rh, rl), (ih, il) = split(M.real), split(M.imag)
    return rh + 1j * ih, rl + 1j * il


def split_product(A, B, cross=("hl", "lh")):
    """A @ B from bf16 parts: hi*hi plus the listed cross terms, result in FP32."""
    Ah, Al = cmat_split(A)
    Bh, Bl = cmat_split(B)
    C = Ah @ Bh
    if "hl" in cross:
        C = C + Ah @ Bl
    if "lh" in cross:
        C = C + Al @ Bh
    return C.real.astype(np.float32).astype(np.float64) + 1j * C.imag.astype(np.float32).astype(np.float64)


def split_sweep(Sa, Sb, cross=("hl", "lh")):
    """<a|b> by the two half-steps per site, every product split."""
    E = np.ones((1, 1), dtype=complex)
    for A, B in zip(Sa, Sb):
        # A, B: (chi_l, 2, chi_r); T_s = E B[:, s, :]; E' = sum_s A[:, s, :]^H T_s
        T = [split_product(E, B[:, s, :], cross) for s in range(2)]
        E = sum(split_product(A[:, s, :].conj().T, T[s], cross) for s in range(2))
    return E[0, 0]


def states(n=60, d=2, count=6, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.6, 1.4, size=(count, n))  # close features: K well above 1e-8
    out = []
    for x in X:
        S = mps.build_mps(x, d, 2, 0.25, 32, 1e-8).sites
        out.append(mps.round_sites(S, "c64"))
    return out


def rel_errors(S, cross=("hl", "lh")):
    errs = []
    for i in range(len(S)):
        for j in range(i + 1, len(S)):
            k64 = abs(overlap.sweep_left_to_right(S[i], S[j])) ** 2
            ks = abs(split_sweep(S[i], S[j], cross)) ** 2
            assert k64 > 1e-8
            errs.append(abs(ks - k64) / k64)
    return np.array(errs)


def test_split_products_stay_inside_the_parity_bar():
    S = states()
    e = rel_errors(S)
    assert np.max(e) < 2e-3
    assert np.median(e) < 2e-4
    assert np.median(e) > 1e-8  # the emulation does round


def test_dropping_a_cross_term_breaks_the_bar():
    S = states(count=4)
    e = rel_errors(S, cross=("hl",))
    assert np.max(e) > 2e-3
