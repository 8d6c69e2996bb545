"""Host-side checks of libqk: it loads, exports every symbol include/qk.h
declares, its schedule length matches the circuit, and bad arguments are
rejected before anything reaches a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2411_09336_gb300", "libqk.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return C.CDLL(LIB)


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qk_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("n,d", [(8, 1), (50, 2), (100, 4), (165, 6), (9, 0), (12, 11)])
def test_schedule_length(lib, n, d):
    from oracle import circuit
    lib.qk_schedule_length.restype = C.c_int64
    assert lib.qk_schedule_length(n, d) == len(circuit.schedule(n, d))


def test_bad_arguments_rejected_on_host(lib):
    import numpy as np
    lib.qk_last_error.restype = C.c_char_p
    X = np.zeros((4, 8))
    out = C.c_void_p()
    f = lib.qk_build_states
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                  C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    cases = [
        dict(n=8, d=8),            # d > n-1
        dict(n=8, d=-1),
        dict(n=1, d=0),            # n < 2
        dict(n=8, d=1, chi=0),
        dict(n=8, d=1, chi=129),
        dict(n=8, d=1, eps=-1.0),
        dict(n=8, d=1, reps=0),
        dict(n=8, d=1, gamma=float("nan")),
    ]
    for c in cases:
        st = f(X.ctypes.data, 4, c["n"], c["d"], c.get("reps", 2), c.get("gamma", 0.5),
               c.get("chi", 16), c.get("eps", 0.0), 1, None, None, C.byref(out))
        assert st == 1, c
        assert lib.qk_last_error()
    # NULL output pointer
    assert f(X.ctypes.data, 4, 8, 1, 2, 0.5, 16, 0.0, 1, None, None, None) == 1


def test_null_handles_rejected_on_host(lib):
    """Entry points taking batches reject NULL handles before any CUDA call."""
    lib.qk_last_error.restype = C.c_char_p
    k, b = C.c_int32(), C.c_int32()
    us = C.c_double()
    lib.qk_tune_split.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    assert lib.qk_tune_split(None, None, 1, None, C.byref(k), C.byref(b), C.byref(us)) == 1
    assert b"NULL" in lib.qk_last_error()
    lib.qk_set_split_schedule.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int32, C.c_int32]
    assert lib.qk_set_split_schedule(None, None, 1, 1, 16) == 1
    lib.qk_gram.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_void_p,
                            C.c_void_p]
    assert lib.qk_gram(None, None, None, 0, 1, 0.0, None, None) == 1
    lib.qk_mps_shape.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.qk_mps_shape(None, None, None) == 1
    # freeing NULL is a no-op
    lib.qk_mps_free.argtypes = [C.c_void_p]
    assert lib.qk_mps_free(None) == 0


def test_non_finite_features_rejected_on_host(lib):
    """A NaN or infinite feature is an argument error found on the host copy
    of X (no state is built)."""
    import numpy as np
    lib.qk_last_error.restype = C.c_char_p
    f = lib.qk_build_states
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                  C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    out = C.c_void_p()
    for bad in (np.nan, np.inf, -np.inf):
        X = np.zeros((3, 6))
        X[2, 4] = bad
        assert f(X.ctypes.data, 3, 6, 1, 2, 0.5, 16, 0.0, 1, None, None, C.byref(out)) == 1
        assert b"non-finite" in lib.qk_last_error()
        assert out.value is None
