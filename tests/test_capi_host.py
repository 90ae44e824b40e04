"""CPU-only checks of the C ABI: the library builds, loads, exports every
declared entry point, and rejects bad arguments before touching a GPU."""
import ctypes
import math
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def frr():
    from paper_2501_07642_b300 import build
    build.build_library()
    from paper_2501_07642_b300 import frr as f
    return f


def _declared_functions():
    text = (ROOT / "include" / "frr.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(frr_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(frr):
    names = _declared_functions()
    assert "frr_init" in names and "frr_select" in names and "frr_randtest" in names
    lib = ctypes.CDLL(str(frr.LIB_PATH))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_strerror(frr):
    o = frr.frr_default_opts()
    assert (o.precision, o.whiten, o.ridge, o.band_safety) == (frr.FRR_SPLIT_BF16, frr.FRR_CHOL, 0.1, 2.0)
    assert o.prep == frr.FRR_PREP_TENSOR and o.autotune == 0
    assert o.cuda_stream is None
    for code in frr.STATUS:
        assert frr.strerror(code)
    assert "degenerate" in frr.strerror(-2)


def _init_status(frr, X, n, d, n1, opts=None):
    h = ctypes.c_void_p()
    X = np.ascontiguousarray(X, dtype=np.float64)
    st = frr.lib().frr_init(ctypes.byref(h), X.ctypes.data, n, d, n1, None if opts is None else ctypes.byref(opts))
    assert not h.value
    return st


def test_init_rejects_bad_arguments_without_a_gpu(frr):
    X = np.random.default_rng(0).standard_normal((10, 3))
    assert _init_status(frr, X, 1, 3, 1) == -1           # n < 2
    assert _init_status(frr, X, 10, 0, 5) == -1          # d < 1
    assert _init_status(frr, X, 10, 3, 0) == -1          # n1 < 1
    assert _init_status(frr, X, 10, 3, 10) == -1         # n1 > n - 1
    Xn = X.copy(); Xn[3, 1] = math.nan
    assert _init_status(frr, Xn, 10, 3, 5) == -1         # non-finite X
    Xi = X.copy(); Xi[0, 0] = math.inf
    assert _init_status(frr, Xi, 10, 3, 5) == -1
    Xw = np.random.default_rng(1).standard_normal((10, 9))
    assert _init_status(frr, Xw, 10, 9, 5) == -2         # d >= n - 1 under Cholesky whitening
    big = np.zeros((2049, 1))
    assert _init_status(frr, big, 2049, 1, 1000) == -9   # beyond the compiled shapes
    o = frr.frr_default_opts(); o.precision = 7
    assert _init_status(frr, X, 10, 3, 5, o) == -1
    o = frr.frr_default_opts(); o.whiten = frr.FRR_RIDGE; o.ridge = 0.0
    assert _init_status(frr, X, 10, 3, 5, o) == -1
    o = frr.frr_default_opts(); o.band_safety = 0.5
    assert _init_status(frr, X, 10, 3, 5, o) == -1
    o = frr.frr_default_opts(); o.prep = 2
    assert _init_status(frr, X, 10, 3, 5, o) == -1


def test_null_context_is_rejected(frr):
    L = frr.lib()
    K = ctypes.c_int64()
    assert L.frr_balance(None, 1, 0, 10, None) == -1
    assert L.frr_select(None, 1, 0, 10, 0.1, math.nan, None, None, 0, ctypes.byref(K)) == -1
    assert L.frr_stream_chunk(None, 0, 1) == -1
    assert L.frr_last_stats(None, None) == -1
    r = frr.frr_tune_result()
    assert L.frr_autotune(None, 0, ctypes.byref(r)) == -1
    assert L.frr_autotune(None, 0, None) == -1
    L.frr_destroy(None)  # ignored


def test_batch_rejects_bad_options_without_a_gpu(frr):
    L = frr.lib()
    ex = (frr.frr_experiment * 1)()
    o = frr.frr_default_opts()
    assert o.autotune == 0
    o.autotune = 2
    st = frr.frr_batch_stats()
    assert L.frr_batch_run(ctypes.addressof(ex), 1, ctypes.byref(o), ctypes.byref(st)) == -1
    assert L.frr_batch_run(None, 1, None, None) == -1
    assert L.frr_batch_run(ctypes.addressof(ex), 0, None, None) == -1


def test_fast_distance_rejects_bad_arguments_without_a_gpu(frr):
    L = frr.lib()
    X = np.zeros((4, 3), dtype=np.float32)
    D = np.zeros((4, 4), dtype=np.float32)
    st = frr.STATUS
    assert st[L.frr_fast_distance(None, 4, None, 0, 3, 0, D.ctypes.data, None)] == "FRR_E_ARG"
    assert st[L.frr_fast_distance(X.ctypes.data, 4, None, 0, 3, 0, None, None)] == "FRR_E_ARG"
    assert st[L.frr_fast_distance(X.ctypes.data, 0, None, 0, 3, 0, D.ctypes.data, None)] == "FRR_E_ARG"
    assert st[L.frr_fast_distance(X.ctypes.data, 4, None, 0, 0, 0, D.ctypes.data, None)] == "FRR_E_ARG"
    assert st[L.frr_fast_distance(X.ctypes.data, 4, X.ctypes.data, 0, 3, 0, D.ctypes.data, None)] == "FRR_E_ARG"
    assert st[L.frr_fast_distance(X.ctypes.data, 1 << 31, None, 0, 3, 0, D.ctypes.data, None)] == "FRR_E_UNSUPPORTED"
