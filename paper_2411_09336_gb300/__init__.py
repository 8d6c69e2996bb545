"""Python binding of libqk (quantum-kernel Gram matrices via MPS on GB300).

Argument marshalling only: every step of the computation runs in libqk's CUDA
kernels.  Functions carry the C names of include/qk.h.  PyTorch provides device
memory and streams; arrays may be numpy arrays (host) or torch tensors (host
or CUDA), passed to the library as raw pointers.

The library must have been built (python -c "import __graft_entry__ as g;
g.build()" or python paper_2411_09336_gb300/build.py); importing this package
without libqk.so raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqk.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqk.so is not built ({LIB_PATH}); run paper_2411_09336_gb300/build.py")

_lib = C.CDLL(LIB_PATH)

QK_OK, QK_ERR_INVALID_ARG, QK_ERR_OOM, QK_ERR_CUDA, QK_ERR_NUMERIC, QK_ERR_TIMEOUT = range(6)
QK_PREC_FP64, QK_PREC_SPLIT_BF16, QK_PREC_SPLIT_BF16X3 = 0, 1, 2
QK_STORE_C128, QK_STORE_C64 = 0, 1
QK_SPLIT_REFINE_ABOVE = 1e-3  # mirrors include/qk.h
_PREC = {"fp64": QK_PREC_FP64, "split": QK_PREC_SPLIT_BF16, "split_bf16": QK_PREC_SPLIT_BF16,
         "split_bf16x3": QK_PREC_SPLIT_BF16X3}
_STORE = {"c128": QK_STORE_C128, "c64": QK_STORE_C64}

_vp, _i32, _i64, _f64, _f32, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float, C.c_uint64


def _sig(name, args, res=C.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("qk_last_error", [], C.c_char_p)
_sig("qk_schedule_length", [_i32, _i32], _i64)
_sig("qk_build_states", [_vp, _i64, _i32, _i32, _i32, _f64, _i32, _f64, C.c_int, _vp, _vp, C.POINTER(_vp)])
_sig("qk_mps_import", [_i64, _i32, _vp, _vp, C.c_int, _vp, C.POINTER(_vp)])
_sig("qk_mps_shape", [_vp, C.POINTER(_i64), C.POINTER(_i32)])
_sig("qk_mps_bond_dims", [_vp, _vp])
_sig("qk_mps_trunc_weight", [_vp, _vp])
_sig("qk_mps_bytes", [_vp, C.POINTER(_i64)])
_sig("qk_mps_export", [_vp, _i64, _vp, _i64])
_sig("qk_mps_free", [_vp])
_sig("qk_gram", [_vp, _vp, _vp, _i64, C.c_int, _f64, _vp, C.POINTER(_i64)])
_sig("qk_gram_pairs", [_vp, _vp, _vp, _i64, _vp, C.c_int, _vp])
_sig("qk_mps_rz_copies", [_vp, _vp, _i64, _vp, C.POINTER(_vp)])
_sig("qk_mps_blob_bytes", [_vp, C.POINTER(_i64)])
_sig("qk_mps_save", [_vp, _vp, _i64])
_sig("qk_mps_load", [_vp, _i64, _vp, C.POINTER(_vp)])
_sig("qk_last_profile", [C.POINTER(_f64), C.POINTER(_f64), C.POINTER(_f64)])
_sig("qk_last_build_profile", [C.POINTER(_f64), _vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64),
                               C.POINTER(_f64)])
_sig("qk_gram_pairs_noalloc", [_vp, _vp, _vp, _i64, _vp, _vp])
_sig("qk_debug_stall_next_split", [_i32])
_sig("qk_debug_tc_profile", [_i32])
_sig("qk_debug_tc_max_ctas", [_i32])
_sig("qk_debug_tc_variant", [_i32])
_sig("qk_last_tc_profile", [_vp, C.POINTER(_i32)])
_sig("qk_tune_split", [_vp, _vp, C.c_int, _vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_f64)])
_sig("qk_set_split_schedule", [_vp, _vp, C.c_int, _i32, _i32])


class QKError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.qk_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != QK_OK:
        raise QKError(st, where)


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (which must stay alive)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    ptr = getattr(a, "data_ptr", None)
    if ptr is not None:
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as_f64(X):
    if isinstance(X, np.ndarray):
        return np.ascontiguousarray(X, dtype=np.float64)
    import torch
    return X.to(torch.float64).contiguous()


def qk_schedule_length(n: int, d: int) -> int:
    return int(_lib.qk_schedule_length(n, d))


class MPSBatch:
    """Handle of a library-owned batch of MPS states (qk_mps_batch*)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)
        N = _i64()
        n = _i32()
        _check(_lib.qk_mps_shape(self._h, C.byref(N), C.byref(n)), "qk_mps_shape")
        self.N, self.n = N.value, n.value

    @property
    def handle(self):
        return self._h

    def bond_dims(self) -> np.ndarray:
        out = np.zeros((self.N, self.n + 1), dtype=np.int32)
        _check(_lib.qk_mps_bond_dims(self._h, out.ctypes.data), "qk_mps_bond_dims")
        return out

    def trunc_weight(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.float64)
        _check(_lib.qk_mps_trunc_weight(self._h, out.ctypes.data), "qk_mps_trunc_weight")
        return out

    def nbytes(self) -> int:
        b = _i64()
        _check(_lib.qk_mps_bytes(self._h, C.byref(b)), "qk_mps_bytes")
        return b.value

    def export(self, s: int) -> list:
        """State s as a list of site tensors A_k[a, q, b] (complex128)."""
        dims = self.bond_dims()[s]
        cap = int(sum(4 * dims[k] * dims[k + 1] for k in range(self.n)))
        buf = np.zeros(cap, dtype=np.float64)
        _check(_lib.qk_mps_export(self._h, s, buf.ctypes.data, cap), "qk_mps_export")
        z = buf[0::2] + 1j * buf[1::2]
        out, o = [], 0
        for k in range(self.n):
            cnt = 2 * dims[k] * dims[k + 1]
            out.append(z[o:o + cnt].reshape(dims[k], 2, dims[k + 1]))
            o += cnt
        return out

    def free(self):
        if self._h is not None and self._h.value:
            _lib.qk_mps_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qk_build_states(X, d: int, reps: int, gamma: float, chi_max: int, eps: float,
                    store: str = "c64", rank_trace=None, stream=None) -> MPSBatch:
    """Simulate every row of X (N x n, host or device) as an MPS (qk.h)."""
    X = _as_f64(X)
    N, n = X.shape
    h = _vp()
    _check(_lib.qk_build_states(_ptr(X), N, n, d, reps, float(gamma), chi_max, float(eps),
                                _STORE[store], _ptr(rank_trace), _stream_ptr(stream), C.byref(h)),
           "qk_build_states")
    return MPSBatch(h.value)


def qk_mps_import(states: list, store: str = "c64", stream=None) -> MPSBatch:
    """Wrap a list of MPS (each a list of (chi_k, 2, chi_k+1) arrays) as a batch."""
    N = len(states)
    n = len(states[0])
    dims = np.zeros((N, n + 1), dtype=np.int32)
    flat = []
    for s, st in enumerate(states):
        dims[s, 0] = 1
        for k, A in enumerate(st):
            dims[s, k + 1] = A.shape[2]
            z = np.ascontiguousarray(A, dtype=np.complex128).reshape(-1)
            flat.append(np.stack([z.real, z.imag], axis=1).reshape(-1))
    buf = np.ascontiguousarray(np.concatenate(flat))
    h = _vp()
    _check(_lib.qk_mps_import(N, n, dims.ctypes.data, buf.ctypes.data, _STORE[store],
                              _stream_ptr(stream), C.byref(h)), "qk_mps_import")
    return MPSBatch(h.value)


def qk_gram(A: MPSBatch, B: MPSBatch | None = None, prec: str = "fp64", refine_floor: float = 0.0,
            out=None, stream=None):
    """Gram block K[i, j] = |<a_i|b_j>|^2 (B None or B is A: symmetric).

    Returns (K, n_refined); K is `out` if given (numpy or torch, host or
    device, float64, shape (N_A, N_B)), else a new CUDA torch tensor."""
    import torch
    sym = B is None or B is A
    B = A if sym else B
    if out is None:
        out = torch.empty((A.N, B.N), dtype=torch.float64, device="cuda")
    nref = _i64()
    _check(_lib.qk_gram(A.handle, B.handle, _ptr(out), B.N, _PREC[prec], float(refine_floor),
                        _stream_ptr(stream), C.byref(nref)), "qk_gram")
    return out, nref.value


def _check_pairs(pairs, where: str, cuda_only: bool = False):
    """pairs must be int32 of shape (P, 2) (a CUDA tensor when cuda_only)."""
    dt = getattr(pairs, "dtype", None)
    ok_dtype = dt == np.int32 or str(dt) == "torch.int32"
    if not ok_dtype or len(pairs.shape) != 2 or pairs.shape[1] != 2:
        raise ValueError(f"{where}: pairs must be int32 of shape (P, 2), got {dt} {tuple(pairs.shape)}")
    if cuda_only and not getattr(pairs, "is_cuda", False):
        raise ValueError(f"{where}: pairs must be a CUDA tensor")


def _check_out(out, P: int, where: str, cuda_only: bool = False):
    """out must be float64 with at least P elements (a CUDA tensor when cuda_only)."""
    dt = getattr(out, "dtype", None)
    if not (dt == np.float64 or str(dt) == "torch.float64"):
        raise ValueError(f"{where}: out must be float64, got {dt}")
    numel = out.size if isinstance(out, np.ndarray) else out.numel()
    if numel < P:
        raise ValueError(f"{where}: out holds {numel} values, {P} needed")
    if cuda_only and not getattr(out, "is_cuda", False):
        raise ValueError(f"{where}: out must be a CUDA tensor")


def qk_gram_pairs(A: MPSBatch, B: MPSBatch, pairs, prec: str = "fp64", out=None, stream=None):
    """K[p] = |<a_{pairs[p,0]}|b_{pairs[p,1]}>|^2; pairs int32 (P, 2)."""
    import torch
    if isinstance(pairs, np.ndarray):
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    _check_pairs(pairs, "qk_gram_pairs")
    P = pairs.shape[0]
    if out is None:
        out = torch.empty(P, dtype=torch.float64, device="cuda")
    _check_out(out, P, "qk_gram_pairs")
    _check(_lib.qk_gram_pairs(A.handle, B.handle, _ptr(pairs), P, _ptr(out), _PREC[prec],
                              _stream_ptr(stream)), "qk_gram_pairs")
    return out


def qk_mps_rz_copies(src: MPSBatch, phi, stream=None) -> MPSBatch:
    """Copies of every state with a final exp(-i sum_k phi[c, k] Z_k) layer;
    phi (copies, n) float64; output state c * N + s."""
    phi = _as_f64(phi)
    h = _vp()
    _check(_lib.qk_mps_rz_copies(src.handle, _ptr(phi), phi.shape[0], _stream_ptr(stream), C.byref(h)),
           "qk_mps_rz_copies")
    return MPSBatch(h.value)


def qk_mps_blob_bytes(b: MPSBatch) -> int:
    n = _i64()
    _check(_lib.qk_mps_blob_bytes(b.handle, C.byref(n)), "qk_mps_blob_bytes")
    return n.value


def qk_mps_save(b: MPSBatch, blob) -> None:
    """Serialise into `blob` (numpy uint8 / torch uint8, host or device)."""
    nbytes = blob.nbytes if isinstance(blob, np.ndarray) else blob.numel() * blob.element_size()
    _check(_lib.qk_mps_save(b.handle, _ptr(blob), nbytes), "qk_mps_save")


def qk_mps_load(blob, stream=None) -> MPSBatch:
    nbytes = blob.nbytes if isinstance(blob, np.ndarray) else blob.numel() * blob.element_size()
    h = _vp()
    _check(_lib.qk_mps_load(_ptr(blob), nbytes, _stream_ptr(stream), C.byref(h)), "qk_mps_load")
    return MPSBatch(h.value)


def qk_last_profile() -> dict:
    """Device milliseconds of the last qk_gram / qk_gram_pairs call."""
    a, b, c = _f64(), _f64(), _f64()
    _check(_lib.qk_last_profile(C.byref(a), C.byref(b), C.byref(c)), "qk_last_profile")
    return {"overlap_ms": a.value, "refine_ms": b.value, "total_ms": c.value}


def qk_debug_stall_next_split(on: bool = True) -> None:
    """Test hook: the next tensor-core overlap launch lets one bounded wait run
    out (the call then fails with QK_ERR_TIMEOUT; see include/qk.h)."""
    _check(_lib.qk_debug_stall_next_split(1 if on else 0), "qk_debug_stall_next_split")


TC_PHASES = ("issue", "wait_copies", "wait_ring", "wait_mma", "epilogue", "barrier", "gemms", "chunks", "tiles",
             "topup", "mma")


def qk_debug_tc_profile(on: bool = True) -> None:
    """Profiling switch of the tensor-core overlap kernel (see include/qk.h)."""
    _check(_lib.qk_debug_tc_profile(1 if on else 0), "qk_debug_tc_profile")


def qk_debug_tc_max_ctas(ctas: int = 0) -> None:
    """Test knob: cap the tensor-core kernel's grid (0: default)."""
    _check(_lib.qk_debug_tc_max_ctas(int(ctas)), "qk_debug_tc_max_ctas")


def qk_debug_tc_variant(flags: int) -> None:
    """Operand-stream variant of the tensor-core kernel (bits: 1 GEMM-block L2
    prefetch, 2 next-site L2 prefetch, 4 normal L2 priority for the static
    operands, 8 drop consumed scratch lines without write-back; see
    include/qk.h)."""
    _check(_lib.qk_debug_tc_variant(int(flags)), "qk_debug_tc_variant")


def qk_last_tc_profile() -> dict:
    """Cycle counters by phase of the last profiled tensor-core launch."""
    v = np.zeros(len(TC_PHASES), dtype=np.float64)
    ctas = _i32()
    _check(_lib.qk_last_tc_profile(v.ctypes.data, C.byref(ctas)), "qk_last_tc_profile")
    out = dict(zip(TC_PHASES, v.tolist()))
    out["ctas"] = ctas.value
    return out


BUILD_PHASES = ("theta", "qr", "jacobi", "factors_out", "moves", "other")


def qk_last_build_profile() -> dict:
    """Device profile of the last qk_build_states call: kernel milliseconds,
    SM-milliseconds per phase (summed over CTAs), Jacobi sweeps and
    factorisations."""
    ms = _f64()
    ph = np.zeros(len(BUILD_PHASES), dtype=np.float64)
    ctas, sw, nf, fl = _i64(), _i64(), _i64(), _f64()
    _check(_lib.qk_last_build_profile(C.byref(ms), ph.ctypes.data, C.byref(ctas), C.byref(sw), C.byref(nf),
                                      C.byref(fl)), "qk_last_build_profile")
    return {"kernel_ms": ms.value, "phase_sm_ms": dict(zip(BUILD_PHASES, ph.tolist())), "ctas": ctas.value,
            "sweeps": sw.value, "factorisations": nf.value, "fp64_flops": fl.value}


def qk_gram_pairs_noalloc(A: MPSBatch, B: MPSBatch, pairs, out, stream=None):
    """FP64 pair overlaps into the caller's device buffer `out` with no
    allocation inside the library call (bond dimensions <= 64; pairs and out
    must be CUDA tensors).  See include/qk.h for the shared-scratch rules."""
    _check_pairs(pairs, "qk_gram_pairs_noalloc", cuda_only=True)
    _check_out(out, pairs.shape[0], "qk_gram_pairs_noalloc", cuda_only=True)
    _check(_lib.qk_gram_pairs_noalloc(A.handle, B.handle, _ptr(pairs), pairs.shape[0], _ptr(out),
                                      _stream_ptr(stream)), "qk_gram_pairs_noalloc")
    return out



def qk_tune_split(A: MPSBatch, B: MPSBatch | None = None, prec: str = "split", stream=None) -> dict:
    """Tile schedule of the split Gram of (A, B) chosen by timing candidates on
    a sample (cached; a cached or set schedule is returned as is)."""
    B = A if B is None else B
    k, b, us = _i32(), _i32(), _f64()
    _check(_lib.qk_tune_split(A.handle, B.handle, _PREC[prec], _stream_ptr(stream), C.byref(k), C.byref(b),
                              C.byref(us)), "qk_tune_split")
    return {"kets_per_tile": k.value, "band": b.value, "us_per_pair": us.value}


def qk_set_split_schedule(A: MPSBatch, B: MPSBatch | None = None, prec: str = "split", kets_per_tile: int = 4,
                          band: int = 16) -> None:
    B = A if B is None else B
    _check(_lib.qk_set_split_schedule(A.handle, B.handle, _PREC[prec], int(kets_per_tile), int(band)),
           "qk_set_split_schedule")

_sig("qk_surrogate_create", [_i32, _i32, _u64, C.POINTER(_vp)])
_sig("qk_surrogate_free", [_vp])
_sig("qk_surrogate_param_count", [_vp], _i64)
_sig("qk_surrogate_get_params", [_vp, _vp])
_sig("qk_surrogate_set_params", [_vp, _vp])
_sig("qk_surrogate_set_bf16", [_vp, _i32])
_sig("qk_surrogate_set_target_scale", [_vp, _f64, _f64])
_sig("qk_surrogate_loss_grad", [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _i64, _vp, C.POINTER(_f64), _vp])
_sig("qk_surrogate_train", [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _i64, _i32, _i32, _f32, _u64, _vp,
                            C.POINTER(_f64)])
_sig("qk_surrogate_predict", [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _i64, _vp, _vp])
_sig("qk_surrogate_calibrate", [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _i64, _f64, _i32, _vp])
_sig("qk_surrogate_bins", [_vp, C.POINTER(_i32), _vp, _vp])
_sig("qk_gram_surrogate", [_vp, _vp, _vp, _vp, _vp, _f64, _vp, _i64, _vp, C.c_int, _vp, C.POINTER(_i64)])


class Surrogate:
    """Handle of the library's MLP surrogate for log K (qk_surrogate*)."""

    def __init__(self, in_dim: int, hidden: int = 512, seed: int = 0):
        h = _vp()
        _check(_lib.qk_surrogate_create(in_dim, hidden, seed, C.byref(h)), "qk_surrogate_create")
        self._h = h
        self.in_dim, self.hidden = in_dim, hidden

    @property
    def handle(self):
        return self._h

    def param_count(self) -> int:
        return int(_lib.qk_surrogate_param_count(self._h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(_lib.qk_surrogate_get_params(self._h, out.ctypes.data), "qk_surrogate_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.qk_surrogate_set_params(self._h, p.ctypes.data), "qk_surrogate_set_params")

    def set_bf16(self, on: bool):
        _check(_lib.qk_surrogate_set_bf16(self._h, 1 if on else 0), "qk_surrogate_set_bf16")

    def set_target_scale(self, mean: float, scale: float):
        _check(_lib.qk_surrogate_set_target_scale(self._h, float(mean), float(scale)), "qk_surrogate_set_target_scale")

    def loss_grad(self, Xa, Xb, pairs, target, stream=None):
        Xa, Xb = _as_f64(Xa), _as_f64(Xb)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        target = _as_f64(target)
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = _f64()
        _check(_lib.qk_surrogate_loss_grad(self._h, _ptr(Xa), Xa.shape[0], _ptr(Xb), Xb.shape[0], Xa.shape[1],
                                           _ptr(pairs), _ptr(target), len(pairs), g.ctypes.data, C.byref(loss),
                                           _stream_ptr(stream)), "qk_surrogate_loss_grad")
        return loss.value, g

    def train(self, Xa, Xb, pairs, target, epochs=10, batch=2048, lr=1e-3, seed=0, stream=None) -> float:
        Xa, Xb = _as_f64(Xa), _as_f64(Xb)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        target = _as_f64(target)
        loss = _f64()
        _check(_lib.qk_surrogate_train(self._h, _ptr(Xa), Xa.shape[0], _ptr(Xb), Xb.shape[0], Xa.shape[1],
                                       _ptr(pairs), _ptr(target), len(pairs), epochs, batch, float(lr), seed,
                                       _stream_ptr(stream), C.byref(loss)), "qk_surrogate_train")
        return loss.value

    def predict(self, Xa, Xb, pairs, stream=None) -> np.ndarray:
        Xa, Xb = _as_f64(Xa), _as_f64(Xb)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        y = np.zeros(len(pairs))
        _check(_lib.qk_surrogate_predict(self._h, _ptr(Xa), Xa.shape[0], _ptr(Xb), Xb.shape[0], Xa.shape[1],
                                         _ptr(pairs), len(pairs), y.ctypes.data, _stream_ptr(stream)),
               "qk_surrogate_predict")
        return y

    def calibrate(self, Xa, Xb, pairs, truth, alpha=0.05, n_bins=8, stream=None):
        Xa, Xb = _as_f64(Xa), _as_f64(Xb)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        truth = _as_f64(truth)
        _check(_lib.qk_surrogate_calibrate(self._h, _ptr(Xa), Xa.shape[0], _ptr(Xb), Xb.shape[0], Xa.shape[1],
                                           _ptr(pairs), _ptr(truth), len(pairs), float(alpha), n_bins,
                                           _stream_ptr(stream)), "qk_surrogate_calibrate")

    def bins(self):
        nb = _i32()
        _check(_lib.qk_surrogate_bins(self._h, C.byref(nb), None, None), "qk_surrogate_bins")
        e = np.zeros(nb.value + 1)
        b = np.zeros(nb.value)
        _check(_lib.qk_surrogate_bins(self._h, C.byref(nb), e.ctypes.data, b.ctypes.data), "qk_surrogate_bins")
        return e, b

    def free(self):
        if self._h is not None and self._h.value:
            _lib.qk_surrogate_free(self._h)
            self._h = _vp(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qk_surrogate_create(in_dim: int, hidden: int = 512, seed: int = 0) -> Surrogate:
    return Surrogate(in_dim, hidden, seed)


def qk_gram_surrogate(net: Surrogate, A: MPSBatch, B: MPSBatch, Xa, Xb, tol: float, prec: str = "split",
                      out=None, stream=None):
    """K block (N_A x N_B) with surrogate predictions where the calibrated
    bound <= tol and exact overlaps elsewhere.  Returns (K, accepted, n)."""
    import torch
    Xa, Xb = _as_f64(Xa), _as_f64(Xb)
    if out is None:
        out = torch.empty((A.N, B.N), dtype=torch.float64, device="cuda")
    acc = torch.empty((A.N, B.N), dtype=torch.uint8, device="cuda")
    na = _i64()
    _check(_lib.qk_gram_surrogate(net.handle, A.handle, B.handle, _ptr(Xa), _ptr(Xb), float(tol), _ptr(out), B.N,
                                  _ptr(acc), _PREC[prec], _stream_ptr(stream), C.byref(na)), "qk_gram_surrogate")
    return out, acc, na.value
