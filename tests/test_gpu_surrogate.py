"""GPU parity of the surrogate's hand-written kernels against the FP64 MLP
oracle, and the accept-or-fall-back Gram on a small workload."""
import numpy as np
import pytest

import workloads
from oracle import mlp, mps, overlap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qk():
    import paper_2411_09336_gb300 as qk
    return qk


def unpack(flat, din, h):
    o = 0
    P = {}
    for k, shape in (("W1", (h, din)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)), ("W3", (1, h)), ("b3", (1,))):
        sz = int(np.prod(shape))
        P[k] = flat[o:o + sz].astype(np.float64).reshape(shape)
        o += sz
    return P


def pack(P):
    return np.concatenate([P[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def small_problem(n=6, N=20, P=57, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(N, n))
    pairs = np.stack([rng.integers(0, N, P), rng.integers(0, N, P)], 1).astype(np.int32)
    t = rng.normal(-5, 2, size=P)
    return X, pairs, t


def test_loss_and_gradients_fp32_vs_oracle(qk):
    n, h = 6, 32
    X, pairs, t = small_problem(n)
    net = qk.qk_surrogate_create(2 * n, h, seed=3)
    net.set_bf16(False)
    rng = np.random.default_rng(1)
    p0 = net.get_params()
    p0[-1] = 0.3
    p0[2 * n * h:2 * n * h + h] = rng.normal(0, 0.1, h)  # nonzero b1
    net.set_params(p0)
    net.set_target_scale(-4.0, 1.5)
    loss, g = net.loss_grad(X, X, pairs, t)
    P = unpack(p0, 2 * n, h)
    F = mlp.pair_features(X, X, pairs)
    L, G = mlp.loss_and_grads(P, F, (t + 4.0) / 1.5)
    assert loss == pytest.approx(L, rel=1e-5)
    gref = pack({k: G[k] for k in G})
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-5


def test_gradients_bf16_vs_oracle(qk):
    n, h = 8, 64
    X, pairs, t = small_problem(n, P=200, seed=2)
    net = qk.qk_surrogate_create(2 * n, h, seed=4)
    p0 = net.get_params()
    loss, g = net.loss_grad(X, X, pairs, t)
    P = unpack(p0, 2 * n, h)
    L, G = mlp.loss_and_grads(P, mlp.pair_features(X, X, pairs), t)
    gref = pack(G)
    assert loss == pytest.approx(L, rel=3e-2)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 3e-2


def test_adam_steps_fp32_vs_oracle(qk):
    n, h = 5, 16
    X, pairs, t = small_problem(n, P=64, seed=5)
    net = qk.qk_surrogate_create(2 * n, h, seed=6)
    net.set_bf16(False)
    p0 = net.get_params()
    net.train(X, X, pairs, t, epochs=2, batch=64, lr=1e-2, seed=0)  # one batch per epoch: order irrelevant
    P = unpack(p0, 2 * n, h)
    m = {k: np.zeros_like(v) for k, v in P.items()}
    v = {k: np.zeros_like(x) for k, x in P.items()}
    F = mlp.pair_features(X, X, pairs)
    for step in (1, 2):
        _, G = mlp.loss_and_grads(P, F, t)
        mlp.adam_step(P, G, m, v, step, 1e-2)
    got = net.get_params()
    assert np.max(np.abs(got - pack(P))) < 2e-5


def test_predict_and_calibration(qk):
    n, h = 6, 32
    X, pairs, t = small_problem(n, N=40, P=3000, seed=7)
    net = qk.qk_surrogate_create(2 * n, h, seed=8)
    net.set_bf16(False)
    y = net.predict(X, X, pairs)
    P = unpack(net.get_params(), 2 * n, h)
    yref, _ = mlp.forward(P, mlp.pair_features(X, X, pairs))
    assert np.max(np.abs(y - yref)) < 1e-4
    net.calibrate(X, X, pairs, t, alpha=0.1, n_bins=4)
    edges, bounds = net.bins()
    ref = mlp.conformal_bounds(y, t, edges, 0.1)
    assert np.allclose(bounds, ref, rtol=0, atol=1e-12)


def test_gram_surrogate_accepts_within_bound_and_falls_back(qk):
    """Train on exact log K of a small workload, calibrate on held-out pairs,
    then build a test x train block: accepted entries come from the network
    and stay within the bound for most of them, the rest equal the exact
    overlaps, and some entries are accepted (the saving)."""
    rng = np.random.default_rng(11)
    n, N, Nt = 10, 160, 40
    X = rng.uniform(-1, 1, size=(N + Nt, n))
    d, reps, gamma = 1, 2, 0.3
    A = qk.qk_build_states(X[:N], d, reps, gamma, 16, 1e-10, store="c128")
    T = qk.qk_build_states(X[N:], d, reps, gamma, 16, 1e-10, store="c128")
    K, _ = qk.qk_gram(A, prec="fp64")
    logK = np.log(K.cpu().numpy())
    iu = np.triu_indices(N, 1)
    allp = np.stack(iu, 1).astype(np.int32)
    sel = rng.permutation(len(allp))
    fit, cal = allp[sel[:9000]], allp[sel[9000:12000]]
    net = qk.qk_surrogate_create(2 * n, 128, seed=1)
    t = logK[fit[:, 0], fit[:, 1]]
    net.set_target_scale(t.mean(), t.std())
    loss = net.train(X[:N], X[:N], fit, t, epochs=60, batch=512, lr=2e-3, seed=2)
    assert loss < 0.2
    net.calibrate(X[:N], X[:N], cal, logK[cal[:, 0], cal[:, 1]], alpha=0.1, n_bins=6)
    tol = 0.5
    Ks, acc, nacc = qk.qk_gram_surrogate(net, T, A, X[N:], X[:N], tol, prec="fp64")
    Kx, _ = qk.qk_gram(T, A, prec="fp64")
    Ks, acc, Kx = Ks.cpu().numpy(), acc.cpu().numpy().astype(bool), Kx.cpu().numpy()
    assert nacc == acc.sum() > 0
    assert np.array_equal(Ks[~acc], Kx[~acc])
    err = np.abs(np.log(Ks[acc]) - np.log(Kx[acc]))
    assert np.mean(err <= tol) >= 0.8


def _bf16(x):
    """Round to bf16 (nearest even) through FP32, as the kernels round GEMM
    operands, and return float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def test_bf16_forward_on_tensor_cores_matches_rounded_reference(qk):
    """bf16 mode runs the layer GEMMs on the tensor cores (tcgen05, bf16
    operands, FP32 accumulation).  Against an FP64 forward pass whose GEMM
    operands are rounded to bf16 the same way, the predictions agree to FP32
    accumulation rounding (several 128 x 128 output tiles, ragged K)."""
    n, h, P = 37, 256, 700
    rng = np.random.default_rng(21)
    X = rng.normal(size=(90, n))
    pairs = np.stack([rng.integers(0, 90, P), rng.integers(0, 90, P)], 1).astype(np.int32)
    net = qk.qk_surrogate_create(2 * n, h, seed=9)
    prm = net.get_params()
    prm[2 * n * h:2 * n * h + h] = rng.normal(0, 0.2, h)
    net.set_params(prm)
    y = net.predict(X, X, pairs)
    Pm = unpack(prm, 2 * n, h)
    F = mlp.pair_features(X, X, pairs).astype(np.float32)
    z1 = _bf16(F) @ _bf16(Pm["W1"]).T + Pm["b1"]
    h1 = np.maximum(z1, 0.0).astype(np.float32)
    z2 = _bf16(h1) @ _bf16(Pm["W2"]).T + Pm["b2"]
    h2 = np.maximum(z2, 0.0).astype(np.float32)
    yref = (_bf16(h2) @ _bf16(Pm["W3"]).T)[:, 0] + Pm["b3"][0]
    scale = np.max(np.abs(yref))
    err = np.abs(y - yref)
    assert np.median(err) <= 1e-5 * scale
    assert np.max(err) <= 2e-3 * scale
