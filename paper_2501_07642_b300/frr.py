"""Thin ctypes binding of libfrr (include/frr.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors to pointers, checks status codes and raises
``FrrError``. If libfrr.so is missing the import fails: there is no fallback.

Host buffers are numpy arrays; device buffers are torch CUDA tensors (their
``data_ptr()`` is passed through). The function names are those of the C ABI.
"""
from __future__ import annotations

import ctypes
import math
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libfrr.so"

FRR_OK = 0
STATUS = {0: "FRR_OK", -1: "FRR_E_ARG", -2: "FRR_E_DEGENERATE", -3: "FRR_E_CUDA", -4: "FRR_E_NOMEM",
          -5: "FRR_E_TIMEOUT", -6: "FRR_E_CAPACITY", -7: "FRR_E_RANGE", -8: "FRR_E_STATE",
          -9: "FRR_E_UNSUPPORTED", -10: "FRR_E_MISMATCH"}
FRR_SPLIT_BF16, FRR_F32 = 0, 1
FRR_CHOL, FRR_RIDGE, FRR_DIAG = 0, 1, 2
FRR_EXACT_SEED = (1 << 64) - 1
PRECISION = {"split_bf16": FRR_SPLIT_BF16, "f32": FRR_F32}
WHITEN = {"chol": FRR_CHOL, "ridge": FRR_RIDGE, "diag": FRR_DIAG}
FRR_PREP_TENSOR, FRR_PREP_FP64_CHAIN = 0, 1
PREP = {"tensor": FRR_PREP_TENSOR, "fp64_chain": FRR_PREP_FP64_CHAIN}


class FrrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name} ({strerror(status)})")


class frr_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("whiten", ctypes.c_int), ("ridge", ctypes.c_double),
                ("band_safety", ctypes.c_double), ("cuda_stream", ctypes.c_void_p), ("autotune", ctypes.c_int),
                ("prep", ctypes.c_int)]


class frr_stats(ctypes.Structure):
    _fields_ = [("draws", ctypes.c_int64), ("candidates", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("threshold_m64", ctypes.c_double), ("band_at_threshold", ctypes.c_double),
                ("max_rel_err", ctypes.c_double), ("max_err_over_band", ctypes.c_double),
                ("boundary_gap_rel", ctypes.c_double), ("parity_at_risk", ctypes.c_int),
                ("band_violations", ctypes.c_int), ("ms_init", ctypes.c_double), ("ms_balance", ctypes.c_double),
                ("ms_select", ctypes.c_double), ("ms_recheck", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class frr_experiment(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("n1", ctypes.c_int64),
                ("whiten", ctypes.c_int), ("ridge", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("first_draw", ctypes.c_uint64), ("B", ctypes.c_uint64), ("q", ctypes.c_double),
                ("threshold", ctypes.c_double), ("keys_out", ctypes.c_void_p), ("M64_out", ctypes.c_void_p),
                ("cap", ctypes.c_int64), ("Y", ctypes.c_void_p), ("tau", ctypes.c_void_p), ("T", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("p_out", ctypes.c_void_p), ("count_out", ctypes.c_void_p),
                ("ci_lo", ctypes.c_double), ("ci_hi", ctypes.c_double), ("K_out", ctypes.c_int64),
                ("status", ctypes.c_int)]


TUNE_MAX = 8


class frr_tune_result(ctypes.Structure):
    _fields_ = [("kb", ctypes.c_int), ("chunks", ctypes.c_int), ("candidates", ctypes.c_int), ("chosen", ctypes.c_int),
                ("ng", ctypes.c_int * TUNE_MAX), ("sb", ctypes.c_int * TUNE_MAX), ("ms", ctypes.c_float * TUNE_MAX)]


class frr_batch_stats(ctypes.Structure):
    _fields_ = [("experiments", ctypes.c_int64), ("draws", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("ms_init", ctypes.c_double), ("ms_balance", ctypes.c_double), ("ms_select", ctypes.c_double)]


class frr_diag_in(ctypes.Structure):
    _fields_ = [("n_T", ctypes.c_int64), ("n_C", ctypes.c_int64), ("d", ctypes.c_int64), ("R2", ctypes.c_double),
                ("sigma", ctypes.c_double), ("q", ctypes.c_double), ("M_obs", ctypes.c_double),
                ("tau", ctypes.c_double), ("alpha", ctypes.c_double), ("power", ctypes.c_double)]


class frr_diag_out(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "k", "sigma2_prog", "rmse_complete", "rmse_realised", "rmse_cs_bound", "c_q", "a_q", "v_a",
        "rmse_accept", "rmse_reduction", "expected_M", "power_at_q", "snr_needed", "q_star", "log10_q_star",
        "c_star", "v_star", "draws_per_accept")] + [("q_star_status", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class frr_stream_info(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("n1", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64), ("total", ctypes.c_uint64),
                ("seen", ctypes.c_uint64), ("q", ctypes.c_double), ("threshold", ctypes.c_double),
                ("K", ctypes.c_int64), ("retained", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise ImportError(f"{LIB_PATH} is not built (python -m paper_2501_07642_b300.build)")
        L = ctypes.CDLL(str(LIB_PATH))
        c = ctypes
        P, U64, I64, D = c.c_void_p, c.c_uint64, c.c_int64, c.c_double
        sig = {
            "frr_default_opts": (None, [P]),
            "frr_strerror": (c.c_char_p, [c.c_int]),
            "frr_init": (c.c_int, [P, P, I64, I64, I64, P]),
            "frr_destroy": (None, [P]),
            "frr_balance": (c.c_int, [P, U64, U64, U64, P]),
            "frr_balance_exact": (c.c_int, [P, U64, U64, P]),
            "frr_select": (c.c_int, [P, U64, U64, U64, D, D, P, P, I64, P]),
            "frr_stream_begin": (c.c_int, [P, U64, D, D, U64]),
            "frr_stream_chunk": (c.c_int, [P, U64, U64]),
            "frr_stream_end": (c.c_int, [P, P, P, I64, P]),
            "frr_assignment": (c.c_int, [P, U64, U64, P]),
            "frr_assignments": (c.c_int, [P, U64, U64, U64, P]),
            "frr_recheck": (c.c_int, [P, U64, P, I64, P]),
            "frr_assignment_from_words": (c.c_int, [P, P, P]),
            "frr_recheck_static": (c.c_int, [P, U64, P, I64, P]),
            "frr_randtest": (c.c_int, [P, U64, P, I64, U64, P, P, I64, D, P, P, P, P]),
            "frr_whitened": (c.c_int, [P, P]),
            "frr_last_stats": (c.c_int, [P, P]),
            "frr_batch_run": (c.c_int, [P, I64, P, P]),
            "frr_autotune": (c.c_int, [P, U64, P]),
            "frr_test_wait_expiry": (c.c_int, [P, U64]),
            "frr_stream_save": (c.c_int, [P, P, c.c_size_t, P]),
            "frr_stream_load": (c.c_int, [P, P, c.c_size_t]),
            "frr_stream_blob_info": (c.c_int, [P, c.c_size_t, P]),
            "frr_diagnose": (c.c_int, [P, P]),
            "frr_fast_distance": (c.c_int, [P, I64, P, I64, I64, c.c_int, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != FRR_OK:
        raise FrrError(st, where)


def strerror(status: int) -> str:
    return lib().frr_strerror(status).decode()


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)!r}")


def frr_default_opts() -> frr_opts:
    o = frr_opts()
    lib().frr_default_opts(ctypes.byref(o))
    return o


class Context:
    """Owns one frr_ctx (frr_init ... frr_destroy)."""

    def __init__(self, X, n1: int, precision: str = "split_bf16", whiten: str = "chol", ridge: float = 0.1,
                 band_safety: float = 2.0, stream=None, prep: str = "tensor"):
        X = np.ascontiguousarray(X, dtype=np.float64)
        n, d = X.shape
        o = frr_default_opts()
        o.precision = PRECISION[precision]
        o.whiten = WHITEN[whiten]
        o.prep = PREP[prep]
        o.ridge = float(ridge)
        o.band_safety = float(band_safety)
        o.cuda_stream = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = ctypes.c_void_p()
        _check(lib().frr_init(ctypes.byref(h), X.ctypes.data, n, d, int(n1), ctypes.byref(o)), "frr_init")
        self.handle = h
        self.n, self.d, self.n1 = n, d, int(n1)
        self.precision, self.whiten = precision, whiten

    def close(self):
        if getattr(self, "handle", None):
            lib().frr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def frr_init(X, n1: int, **kw) -> Context:
    return Context(X, n1, **kw)


def frr_destroy(ctx: Context):
    ctx.close()


def frr_balance(ctx: Context, seed: int, first_draw: int, B: int, M_out=None):
    out = np.empty(B, dtype=np.float32) if M_out is None else M_out
    _check(lib().frr_balance(ctx.handle, seed, first_draw, B, _ptr(out)), "frr_balance")
    return out


def frr_balance_exact(ctx: Context, first_rank: int, B: int, M_out=None):
    out = np.empty(B, dtype=np.float32) if M_out is None else M_out
    _check(lib().frr_balance_exact(ctx.handle, first_rank, B, _ptr(out)), "frr_balance_exact")
    return out


def _q_thr(q, threshold):
    return (math.nan if q is None else float(q)), (math.nan if threshold is None else float(threshold))


def frr_select(ctx: Context, seed: int, first_draw: int, B: int, q=None, threshold=None, cap=None,
               keys_out=None, M64_out=None):
    """Returns (keys, M64) as numpy arrays (or the given output buffers, trimmed)."""
    qq, tt = _q_thr(q, threshold)
    if cap is None:
        cap = B if keys_out is None else len(keys_out)
    keys = np.empty(cap, dtype=np.uint64) if keys_out is None else keys_out
    m64 = np.empty(cap, dtype=np.float64) if M64_out is None else M64_out
    K = ctypes.c_int64()
    _check(lib().frr_select(ctx.handle, seed, first_draw, B, qq, tt, _ptr(keys), _ptr(m64), cap, ctypes.byref(K)),
           "frr_select")
    k = K.value
    if k == len(keys) and k == len(m64):
        return keys, m64  # already exactly K long (slicing a device tensor costs microseconds)
    return keys[:k], m64[:k]


def frr_stream_begin(ctx: Context, seed: int, B_total: int, q=None, threshold=None):
    qq, tt = _q_thr(q, threshold)
    _check(lib().frr_stream_begin(ctx.handle, seed, qq, tt, B_total), "frr_stream_begin")


def frr_stream_chunk(ctx: Context, first_draw: int, B_chunk: int):
    _check(lib().frr_stream_chunk(ctx.handle, first_draw, B_chunk), "frr_stream_chunk")


def frr_stream_end(ctx: Context, cap: int):
    keys = np.empty(cap, dtype=np.uint64)
    m64 = np.empty(cap, dtype=np.float64)
    K = ctypes.c_int64()
    _check(lib().frr_stream_end(ctx.handle, _ptr(keys), _ptr(m64), cap, ctypes.byref(K)), "frr_stream_end")
    return keys[:K.value], m64[:K.value]


def frr_assignment(ctx: Context, seed: int, key: int, w_out=None):
    w = np.empty(ctx.n, dtype=np.uint8) if w_out is None else w_out
    _check(lib().frr_assignment(ctx.handle, seed, key, _ptr(w)), "frr_assignment")
    return w


def frr_stream_save(ctx: Context) -> bytes:
    """The running stream's checkpoint blob (layout in include/frr.h)."""
    size = ctypes.c_size_t()
    st = lib().frr_stream_save(ctx.handle, None, 0, ctypes.byref(size))
    if st != -6:
        _check(st, "frr_stream_save")
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().frr_stream_save(ctx.handle, buf, size.value, ctypes.byref(size)), "frr_stream_save")
    return buf.raw[:size.value]


def frr_stream_load(ctx: Context, blob: bytes):
    _check(lib().frr_stream_load(ctx.handle, blob, len(blob)), "frr_stream_load")


def frr_stream_blob_info(blob: bytes) -> dict:
    info = frr_stream_info()
    _check(lib().frr_stream_blob_info(blob, len(blob), ctypes.byref(info)), "frr_stream_blob_info")
    return info.as_dict()


def frr_assignments(ctx: Context, seed: int, first_draw: int, count: int, w_out=None):
    w = np.empty((count, ctx.n), dtype=np.uint8) if w_out is None else w_out
    _check(lib().frr_assignments(ctx.handle, seed, first_draw, count, _ptr(w)), "frr_assignments")
    return w


def frr_assignment_from_words(ctx: Context, words, w_out=None):
    wd = np.ascontiguousarray(words, dtype=np.uint32) if isinstance(words, (list, tuple, np.ndarray)) else words
    w = np.empty(ctx.n, dtype=np.uint8) if w_out is None else w_out
    _check(lib().frr_assignment_from_words(ctx.handle, _ptr(wd), _ptr(w)), "frr_assignment_from_words")
    return w


def frr_recheck(ctx: Context, seed: int, draws, M64_out=None):
    dr = np.ascontiguousarray(draws, dtype=np.uint64) if isinstance(draws, (list, tuple, np.ndarray)) else draws
    out = np.empty(len(dr), dtype=np.float64) if M64_out is None else M64_out
    _check(lib().frr_recheck(ctx.handle, seed, _ptr(dr), len(dr), _ptr(out)), "frr_recheck")
    return out


def frr_randtest(ctx: Context, seed: int, keys, obs_key: int, Y, tau, alpha: float = 0.05):
    """Returns dict(p, count, ci_lo, ci_hi)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64) if isinstance(keys, (list, tuple, np.ndarray)) else keys
    Y = np.ascontiguousarray(Y, dtype=np.float64) if isinstance(Y, (list, tuple, np.ndarray)) else Y
    tau = np.ascontiguousarray(tau, dtype=np.float64) if isinstance(tau, (list, tuple, np.ndarray)) else tau
    T = len(tau)
    p = np.empty(T, dtype=np.float64)
    cnt = np.empty(T, dtype=np.int64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().frr_randtest(ctx.handle, seed, _ptr(keys), len(keys), obs_key, _ptr(Y), _ptr(tau), T, alpha,
                              _ptr(p), _ptr(cnt), ctypes.byref(lo), ctypes.byref(hi)), "frr_randtest")
    return {"p": p, "count": cnt, "ci_lo": lo.value, "ci_hi": hi.value}


def frr_whitened(ctx: Context):
    z = np.empty((ctx.n, ctx.d), dtype=np.float64)
    _check(lib().frr_whitened(ctx.handle, z.ctypes.data), "frr_whitened")
    return z


def frr_last_stats(ctx: Context) -> dict:
    s = frr_stats()
    _check(lib().frr_last_stats(ctx.handle, ctypes.byref(s)), "frr_last_stats")
    return s.as_dict()


def frr_autotune(ctx: Context, B_probe: int = 0) -> dict:
    """Times the compiled configurations of the split-BF16 balance kernel for this context's
    shape class and makes the fastest the one used from now on (process-wide)."""
    r = frr_tune_result()
    _check(lib().frr_autotune(ctx.handle, int(B_probe), ctypes.byref(r)), "frr_autotune")
    c = r.candidates
    return {"kb": r.kb, "chunks": r.chunks, "chosen": r.chosen, "ng": list(r.ng[:c]), "sb": list(r.sb[:c]),
            "ms": list(r.ms[:c])}


def frr_test_wait_expiry(ctx: Context, wait_cycles: int) -> int:
    """Failure-path test: one balance launch whose covariate tiles never arrive, with every
    bounded wait limited to wait_cycles SM cycles. Returns the raw status (FRR_E_TIMEOUT
    expected) instead of raising."""
    return int(lib().frr_test_wait_expiry(ctx.handle, int(wait_cycles)))


def frr_batch_run(experiments, precision: str = "split_bf16", band_safety: float = 2.0, stream=None,
                  autotune: bool = False, prep: str = "tensor"):
    """experiments: list of dicts with keys X, n1, seed, B (and optional first_draw, q or
    threshold, whiten, ridge, Y, tau, alpha). Returns (list of result dicts, stats dict).
    Outputs are host numpy arrays. autotune: time the kernel configurations on a probe of
    the batch first (cached per shape class)."""
    E = len(experiments)
    arr = (frr_experiment * E)()
    keep = []
    outs = []
    for e, x in enumerate(experiments):
        X = np.ascontiguousarray(x["X"], dtype=np.float64)
        keep.append(X)
        q = x.get("q")
        thr = x.get("threshold")
        B = int(x["B"])
        cap = int(x.get("cap", B))
        keys = np.zeros(cap, dtype=np.uint64)
        m64 = np.zeros(cap, dtype=np.float64)
        o = {"keys": keys, "m64": m64}
        a = arr[e]
        a.X = X.ctypes.data
        a.n, a.d = X.shape
        a.n1 = int(x["n1"])
        a.whiten = WHITEN[x.get("whiten", "chol")]
        a.ridge = float(x.get("ridge", 0.1))
        a.seed = int(x["seed"])
        a.first_draw = int(x.get("first_draw", 0))
        a.B = B
        a.q = math.nan if q is None else float(q)
        a.threshold = math.nan if thr is None else float(thr)
        a.keys_out = keys.ctypes.data
        a.M64_out = m64.ctypes.data
        a.cap = cap
        if x.get("Y") is not None:
            Y = np.ascontiguousarray(x["Y"], dtype=np.float64)
            tau = np.ascontiguousarray(x["tau"], dtype=np.float64)
            p = np.zeros(tau.size)
            cnt = np.zeros(tau.size, dtype=np.int64)
            keep += [Y, tau]
            a.Y, a.tau, a.T = Y.ctypes.data, tau.ctypes.data, tau.size
            a.alpha = float(x.get("alpha", 0.05))
            a.p_out, a.count_out = p.ctypes.data, cnt.ctypes.data
            o.update(p=p, count=cnt)
        outs.append(o)
    opts = frr_default_opts()
    opts.precision = PRECISION[precision]
    opts.band_safety = float(band_safety)
    opts.cuda_stream = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    opts.autotune = 1 if autotune else 0
    opts.prep = PREP[prep]
    st = frr_batch_stats()
    rc = lib().frr_batch_run(ctypes.addressof(arr), E, ctypes.byref(opts), ctypes.byref(st))
    res = []
    for e in range(E):
        a = arr[e]
        o = outs[e]
        K = a.K_out
        r = {"status": a.status, "K": K, "keys": o["keys"][:K], "m64": o["m64"][:K], "ci_lo": a.ci_lo,
             "ci_hi": a.ci_hi}
        if "p" in o:
            r.update(p=o["p"], count=o["count"])
        res.append(r)
    stats = {k: getattr(st, k) for k, _ in frr_batch_stats._fields_}
    stats["status"] = rc
    return res, stats


def frr_diagnose(n_T: int, n_C: int, d: int, R2: float, sigma: float = 1.0, q=None, M_obs=None, tau=None,
                 alpha: float = 0.05, power: float = 0.8) -> dict:
    """Planning diagnostics (realised RMSE from M_obs, ex-ante RMSE at q, q* for tau).
    Host-only; needs no context and no GPU. Outputs that were not asked for are NaN."""
    nan = math.nan
    a = frr_diag_in(int(n_T), int(n_C), int(d), float(R2), float(sigma), nan if q is None else float(q),
                    nan if M_obs is None else float(M_obs), nan if tau is None else float(tau), float(alpha),
                    float(power))
    o = frr_diag_out()
    _check(lib().frr_diagnose(ctypes.byref(a), ctypes.byref(o)), "frr_diagnose")
    return o.as_dict()


def frr_fast_distance(X, Y=None, squared: bool = False, D_out=None, stream=None):
    """Pairwise Euclidean distances between the rows of X (n x d) and Y (m x d), FP32.
    X, Y, D_out: numpy arrays (host) or torch CUDA tensors (device). Returns D_out, or a
    new host array when D_out is None."""
    def _f32(a):
        if hasattr(a, "data_ptr"):
            if a.dtype.__str__() != "torch.float32":
                raise TypeError("device inputs must be float32 tensors")
            return a
        return np.ascontiguousarray(a, dtype=np.float32)
    Xc = _f32(X)
    n, d = Xc.shape
    Yc = None if Y is None else _f32(Y)
    if Yc is not None and Yc.shape[1] != d:
        raise ValueError("X and Y need the same number of columns")
    m = n if Yc is None else Yc.shape[0]
    out = np.empty((n, m), dtype=np.float32) if D_out is None else D_out
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().frr_fast_distance(_ptr(Xc), n, _ptr(Yc), m, d, int(bool(squared)), _ptr(out), st),
           "frr_fast_distance")
    return out
