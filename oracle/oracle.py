"""ctypes front for the FP64 CPU oracle (frr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package. It shares no code
with the CUDA path and does not import it.

``build()`` compiles frr_oracle.c with gcc (-O2 -ffp-contract=off -fopenmp, -mfma where available)
into oracle/_build/libfrr_oracle.so.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "frr_oracle.c"
_OUT = _HERE / "_build" / "libfrr_oracle.so"
_lib = None

WHITEN = {"chol": 0, "ridge": 1, "diag": 2}


def _cpu_has_fma() -> bool:
    try:
        with open("/proc/cpuinfo") as f:
            return any(line.startswith("flags") and " fma " in f" {line.split(':', 1)[1].strip()} " for line in f)
    except OSError:
        return False


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (FP64, no implicit contraction, OpenMP). The explicit
    fma() calls of the preparation are correctly rounded either way; with -mfma they compile
    to the hardware instruction instead of a library call (much faster at n = d = 1000)."""
    _OUT.parent.mkdir(parents=True, exist_ok=True)
    if force or not _OUT.exists() or _OUT.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp.so")
        extra = ["-mfma"] if _cpu_has_fma() else []
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", *extra,
                        "-fPIC", "-shared", str(_SRC), "-o", str(tmp), "-lm"], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        c = ctypes
        P = c.c_void_p
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_unit_words.argtypes = [c.c_uint64, c.c_uint64, c.c_int64, P]
        _lib.oracle_assignment.argtypes = [c.c_uint64, c.c_uint64, c.c_int64, c.c_int64, P]
        _lib.oracle_assignments.argtypes = [c.c_uint64, c.c_uint64, c.c_int64, c.c_int64, c.c_int64, P]
        _lib.oracle_enum_masks.argtypes = [c.c_int64, c.c_int64, c.c_uint64, c.c_int64, P]
        _lib.oracle_enum_masks.restype = c.c_int64
        _lib.oracle_prep.argtypes = [P, c.c_int64, c.c_int64, c.c_int, c.c_double, P, P, P, P]
        _lib.oracle_prep.restype = c.c_int
        _lib.oracle_M.argtypes = [P, c.c_int64, c.c_int64, P]
        _lib.oracle_M.restype = c.c_double
        _lib.oracle_balance.argtypes = [P, c.c_int64, c.c_int64, c.c_int64, c.c_int, c.c_uint64,
                                        c.c_uint64, c.c_int64, P, c.c_int]
        _lib.oracle_balance_list.argtypes = [P, c.c_int64, c.c_int64, c.c_int64, c.c_int, c.c_uint64,
                                             P, c.c_int64, P, c.c_int]
        _lib.oracle_rank_of_mask.argtypes = [c.c_uint64]
        _lib.oracle_rank_of_mask.restype = c.c_uint64
        _lib.oracle_mask_of_rank.argtypes = [c.c_int64, c.c_int64, c.c_uint64]
        _lib.oracle_mask_of_rank.restype = c.c_uint64
        _lib.oracle_distance.argtypes = [P, c.c_int64, P, c.c_int64, c.c_int64, c.c_int, P]
        _lib.oracle_distance_pairs.argtypes = [P, P, c.c_int64, P, c.c_int64, c.c_int, P]
        _lib.oracle_k_from_q.argtypes = [c.c_double, c.c_int64]
        _lib.oracle_k_from_q.restype = c.c_int64
        _lib.oracle_select_from_M.argtypes = [P, c.c_uint64, c.c_int64, c.c_double, c.c_double, P, P, c.c_int64]
        _lib.oracle_select_from_M.restype = c.c_int64
        _lib.oracle_dim.argtypes = [P, P, c.c_int64]
        _lib.oracle_dim.restype = c.c_double
        _lib.oracle_randtest.argtypes = [P, c.c_int64, c.c_int64, P, P, P, c.c_int64, c.c_double,
                                         P, P, P, P, P]
        _lib.oracle_randtest.restype = c.c_int
        _lib.oracle_openmp_threads.restype = c.c_int
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key) -> np.ndarray:
    ctr = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(ctr), _p(k), _p(out))
    return out


def unit_words(seed: int, draw: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    lib().oracle_unit_words(seed, draw, n, _p(out))
    return out


def assignment(seed: int, draw: int, n: int, n1: int) -> np.ndarray:
    w = np.zeros(n, dtype=np.uint8)
    lib().oracle_assignment(seed, draw, n, n1, _p(w))
    return w


def assignments(seed: int, first: int, count: int, n: int, n1: int) -> np.ndarray:
    w = np.zeros((count, n), dtype=np.uint8)
    lib().oracle_assignments(seed, first, count, n, n1, _p(w))
    return w


def enum_masks(n: int, n1: int, first: int = 0, count: int | None = None) -> np.ndarray:
    if count is None:
        count = math.comb(n, n1) - first
    out = np.zeros(max(count, 0), dtype=np.uint64)
    got = lib().oracle_enum_masks(n, n1, first, count, _p(out))
    if got < 0:
        raise ValueError("exact enumeration needs 1 <= n1 <= n <= 63")
    return out[:got]


def rank_of_mask(mask: int) -> int:
    """Colex rank (position in the enumeration order) of an n1-subset mask."""
    return int(lib().oracle_rank_of_mask(int(mask)))


def mask_of_rank(n: int, n1: int, rank: int) -> int:
    """The n1-subset mask at colex rank `rank` (n <= 63)."""
    return int(lib().oracle_mask_of_rank(n, n1, int(rank)))


def masks_to_w(masks: np.ndarray, n: int) -> np.ndarray:
    m = np.asarray(masks, dtype=np.uint64)
    return ((m[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)


def prep(X: np.ndarray, whiten: str = "chol", ridge: float = 0.0):
    """Returns (Zc, L, xbar, S). Raises ValueError on a degenerate factor."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, d = X.shape
    Zc = np.zeros((n, d))
    L = np.zeros((d, d))
    xbar = np.zeros(d)
    S = np.zeros((d, d))
    st = lib().oracle_prep(_p(X), n, d, WHITEN[whiten], float(ridge), _p(Zc), _p(L), _p(xbar), _p(S))
    if st != 0:
        raise ValueError("degenerate covariance: Cholesky pivot below tolerance")
    return Zc, L, xbar, S


def M_of(Zc: np.ndarray, w: np.ndarray) -> float:
    Zc = np.ascontiguousarray(Zc, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.uint8)
    n, d = Zc.shape
    return lib().oracle_M(_p(Zc), n, d, _p(w))


def balance(Zc: np.ndarray, n1: int, seed: int | None, first: int, count: int, threads: int = 0) -> np.ndarray:
    """M for draws [first, first+count); seed=None means exact-enumeration ranks."""
    Zc = np.ascontiguousarray(Zc, dtype=np.float64)
    n, d = Zc.shape
    out = np.zeros(count)
    exact = 1 if seed is None else 0
    lib().oracle_balance(_p(Zc), n, d, n1, exact, 0 if seed is None else seed, first, count, _p(out), threads)
    return out


def balance_list(Zc: np.ndarray, n1: int, seed: int | None, draws, threads: int = 0) -> np.ndarray:
    Zc = np.ascontiguousarray(Zc, dtype=np.float64)
    n, d = Zc.shape
    dr = np.ascontiguousarray(draws, dtype=np.uint64)
    out = np.zeros(dr.size)
    exact = 1 if seed is None else 0
    lib().oracle_balance_list(_p(Zc), n, d, n1, exact, 0 if seed is None else seed, _p(dr), dr.size,
                              _p(out), threads)
    return out


def k_from_q(q: float, B: int) -> int:
    return int(lib().oracle_k_from_q(q, B))


def select_from_M(M: np.ndarray, first: int, q: float | None = None, threshold: float | None = None):
    M = np.ascontiguousarray(M, dtype=np.float64)
    B = M.size
    qq = float("nan") if q is None else float(q)
    tt = float("nan") if threshold is None else float(threshold)
    cap = B
    keys = np.zeros(cap, dtype=np.uint64)
    mo = np.zeros(cap)
    K = lib().oracle_select_from_M(_p(M), first, B, qq, tt, _p(keys), _p(mo), cap)
    return keys[:K].copy(), mo[:K].copy()


def select(Zc: np.ndarray, n1: int, seed: int | None, first: int, B: int, q: float | None = None,
           threshold: float | None = None, threads: int = 0):
    M = balance(Zc, n1, seed, first, B, threads)
    return select_from_M(M, first, q, threshold)


def dim(y: np.ndarray, w: np.ndarray) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.uint8)
    return lib().oracle_dim(_p(y), _p(w), y.size)


def randtest(W: np.ndarray, w_obs: np.ndarray, Y: np.ndarray, tau, alpha: float = 0.05):
    """Returns dict(p, count, near_ties, ci_lo, ci_hi) over the accepted set W (K x n)."""
    W = np.ascontiguousarray(W, dtype=np.uint8)
    K, n = W.shape
    w_obs = np.ascontiguousarray(w_obs, dtype=np.uint8)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    T = tau.size
    p = np.zeros(T)
    cnt = np.zeros(T, dtype=np.int64)
    near = np.zeros(T, dtype=np.int64)
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    lib().oracle_randtest(_p(W), K, n, _p(w_obs), _p(Y), _p(tau), T, alpha, _p(p), _p(cnt), _p(near),
                          ctypes.byref(lo), ctypes.byref(hi))
    return {"p": p, "count": cnt, "near_ties": near, "ci_lo": lo.value, "ci_hi": hi.value}


def threads() -> int:
    return int(lib().oracle_openmp_threads())


def distance(X: np.ndarray, Y: np.ndarray | None = None, squared: bool = False) -> np.ndarray:
    """FP64 pairwise Euclidean distances between the rows of FP32 X (n x d) and Y (m x d)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    Yc = None if Y is None else np.ascontiguousarray(Y, dtype=np.float32)
    m = n if Yc is None else Yc.shape[0]
    out = np.zeros((n, m))
    lib().oracle_distance(_p(X), n, None if Yc is None else _p(Yc), m, d, int(squared), _p(out))
    return out


def distance_pairs(X: np.ndarray, Y: np.ndarray, ij: np.ndarray, squared: bool = False) -> np.ndarray:
    """FP64 distances of the listed (i, j) pairs (an array of shape (count, 2))."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    ij = np.ascontiguousarray(ij, dtype=np.int64)
    out = np.zeros(ij.shape[0])
    lib().oracle_distance_pairs(_p(X), _p(Y), X.shape[1], _p(ij), ij.shape[0], int(squared), _p(out))
    return out
