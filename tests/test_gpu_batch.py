"""GPU parity of the batched driver (one persistent balance launch over many
experiments of uneven n and d) against the FP64 oracle and the single-experiment path."""
import hashlib
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import ar1_covariates, batched_workloads, outcome

pytestmark = pytest.mark.gpu

REL_M64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_07642_b300 import build
    build.build_library()
    O.build()


MIX = [  # (n, d, whiten, B, q, seed)
    (50, 10, "chol", 20_000, 0.01, 11),
    (20, 5, "chol", math.comb(20, 10), 0.05, frr.FRR_EXACT_SEED),
    (137, 60, "chol", 30_000, 0.01, 12),
    (300, 299, "ridge", 25_000, 0.02, 13),
    (513, 100, "chol", 15_000, 0.01, 14),
    (1000, 257, "chol", 12_000, 0.01, 15),
    (2000, 33, "chol", 8_000, 0.01, 16),
    (64, 500, "ridge", 20_000, 0.005, 17),
]


def test_batch_chain_scratch_beyond_its_lent_slice():
    """Each experiment's selection chain takes its scratch from a slice of one block lent by the
    batch; an experiment with K = 1e5 of 2e5 draws needs several MiB (retained sets, recheck
    rows), more than its slice, and takes the rest from the pool. Beside a small experiment,
    both must match the oracle."""
    mix = [(100, 20, "chol", 200_000, 0.5, 21), (60, 12, "ridge", 20_000, 0.01, 22)]
    exps, Xs = [], []
    for k, (n, d, wh, B, q, seed) in enumerate(mix):
        X = ar1_covariates(n, d, 700 + k, 0.3)
        Xs.append(X)
        exps.append(dict(X=X, n1=n // 2, whiten=wh, ridge=0.1, seed=seed, first_draw=5000 * k, B=B, q=q))
    res, stats = frr.frr_batch_run(exps, precision="split_bf16")
    assert stats["status"] == 0 and stats["failed"] == 0
    for k, (x, r) in enumerate(zip(exps, res)):
        n, d, wh, B, q, seed = mix[k]
        assert r["status"] == 0
        Zc, *_ = O.prep(Xs[k], wh, 0.1)
        M = O.balance(Zc, n // 2, seed, x["first_draw"], B)
        wk, wm = O.select_from_M(M, x["first_draw"], q=q)
        assert len(wk) == math.ceil(q * B - 1e-9 * q * B)
        assert np.array_equal(r["keys"], wk), f"experiment {k}"
        assert np.allclose(r["m64"], wm, rtol=REL_M64, atol=0)


@pytest.mark.parametrize("precision,prep", [("split_bf16", "tensor"), ("f32", "tensor"), ("split_bf16", "fp64_chain")])
def test_batch_matches_oracle_and_single_path(precision, prep):
    """Both preparation modes: the batched preparation covers experiments with and without a
    256-column block boundary of the forward substitution (d = 257, 299, 500) in one launch set."""
    exps, Xs = [], []
    for k, (n, d, wh, B, q, seed) in enumerate(MIX):
        X = ar1_covariates(n, d, 500 + k, 0.3)
        Xs.append(X)
        exps.append(dict(X=X, n1=n // 2, whiten=wh, ridge=0.1, seed=seed, first_draw=0 if seed == frr.FRR_EXACT_SEED
                         else 1000 * k, B=B, q=q))
    res, stats = frr.frr_batch_run(exps, precision=precision, prep=prep)
    assert stats["status"] == 0 and stats["failed"] == 0
    for k, (x, r) in enumerate(zip(exps, res)):
        n, d, wh, B, q, seed = MIX[k]
        assert r["status"] == 0
        Zc, *_ = O.prep(Xs[k], wh, 0.1)
        s = None if seed == frr.FRR_EXACT_SEED else seed
        M = O.balance(Zc, n // 2, s, x["first_draw"], B)
        wk, wm = O.select_from_M(M, x["first_draw"], q=q)
        assert np.array_equal(r["keys"], wk), f"experiment {k}"
        assert np.allclose(r["m64"], wm, rtol=REL_M64, atol=0)
        with frr.Context(Xs[k], n // 2, precision=precision, whiten=wh, prep=prep) as ctx:
            sk, sm = frr.frr_select(ctx, seed, x["first_draw"], B, q=q)
        assert np.array_equal(sk, r["keys"]) and np.array_equal(sm, r["m64"])


def test_batch_reports_per_experiment_errors():
    good = dict(X=ar1_covariates(40, 5, 1, 0.0), n1=20, seed=3, B=2000, q=0.05)
    bad = dict(X=ar1_covariates(10, 9, 2, 0.0), n1=5, seed=3, B=2000, q=0.05)  # d >= n - 1 under Cholesky
    res, stats = frr.frr_batch_run([good, bad, good])
    assert stats["status"] == -2 and stats["failed"] == 1
    assert res[0]["status"] == 0 and res[2]["status"] == 0 and res[1]["status"] == -2
    assert np.array_equal(res[0]["keys"], res[2]["keys"]) and res[0]["K"] == 100
    # a non-finite covariate (caught while staging the batch's covariates), a degenerate
    # pivot (a duplicated column: S is singular, found on the device) and an exact-mode rank
    # range beyond C(n, n1) each fail alone
    nan_x = ar1_covariates(40, 5, 4, 0.0)
    nan_x[7, 2] = np.nan
    dup = ar1_covariates(40, 6, 5, 0.0)
    dup[:, 3] = dup[:, 1]
    exact_bad = dict(X=ar1_covariates(12, 3, 6, 0.0), n1=6, seed=frr.FRR_EXACT_SEED, first_draw=900, B=100, q=0.1)
    res, stats = frr.frr_batch_run([good, dict(good, X=nan_x), dict(good, X=dup), exact_bad, good])
    assert [r["status"] for r in res] == [0, -1, -2, -7, 0]
    assert stats["failed"] == 3
    assert np.array_equal(res[0]["keys"], res[4]["keys"])


def _golden_batched():
    path = Path(__file__).resolve().parent / "golden" / "batched_256_accepted.txt"
    rows = {}
    for ln in path.read_text().splitlines():
        if ln and not ln.startswith("#"):
            f = ln.split()
            rows[int(f[0])] = dict(n=int(f[1]), d=int(f[2]), whiten=f[3], K=int(f[4]), sha=f[5], kmin=int(f[6]),
                                   kmax=int(f[7]), ksum=int(f[8]), mmax=float(f[9]))
    return rows


def test_batched_workload_256_experiments_identical_to_oracle():
    """The batched workload: 256 experiments (n log-uniform on [50, 2000], d on [10, 500]),
    1e5 draws each, q = 0.01, in one frr_batch_run. Every experiment's accepted key set must
    be identical to the oracle's over all of its 1e5 draws -- recorded by
    tests/golden/make_batched_golden.py, which calls only the oracle, as a SHA-256 of the
    keys -- and its M64 must agree with the oracle's re-scoring of the accepted keys."""
    gold = _golden_batched()
    wls = batched_workloads(256)
    exps = []
    for w in wls:
        X = w.covariates()
        exps.append(dict(X=X, n1=w.n1, whiten=w.whiten, ridge=w.ridge, seed=w.philox_seed, B=w.draws, q=w.q))
    res, stats = frr.frr_batch_run(exps)
    assert stats["status"] == 0, stats
    differ = []
    for e, (w, r) in enumerate(zip(wls, res)):
        g = gold[e]
        assert (g["n"], g["d"], g["whiten"]) == (w.n, w.d, w.whiten)
        keys = np.ascontiguousarray(r["keys"], dtype="<u8")
        if (len(keys) != g["K"] or hashlib.sha256(keys.tobytes()).hexdigest() != g["sha"]):
            differ.append(e)
    assert not differ, f"accepted sets differ from the oracle in experiments {differ}"
    for e, (w, r) in enumerate(zip(wls, res)):
        Zc, *_ = O.prep(exps[e]["X"], w.whiten, w.ridge)
        got = O.balance_list(Zc, w.n1, w.philox_seed, r["keys"])
        assert np.allclose(r["m64"], got, rtol=REL_M64, atol=0), f"experiment {e}"
        assert math.isclose(float(np.max(r["m64"])), gold[e]["mmax"], rel_tol=REL_M64)


def test_batch_randomization_tests_match_single_path():
    wls = batched_workloads(6)
    exps, Ys = [], []
    for w in wls:
        X = w.covariates()
        with frr.Context(X, w.n1, precision="f32", whiten=w.whiten, ridge=w.ridge) as ctx:
            k0 = frr.frr_select(ctx, w.philox_seed, 0, 20_000, q=w.q)[0][0]
            w_obs = frr.frr_assignment(ctx, w.philox_seed, int(k0))
        Y = outcome(X, w_obs, w.tau_true, w.y_seed, w.noise_sd)
        Ys.append(Y)
        exps.append(dict(X=X, n1=w.n1, whiten=w.whiten, ridge=w.ridge, seed=w.philox_seed, B=20_000, q=w.q, Y=Y,
                         tau=w.tau_grid, alpha=0.05))
    res, stats = frr.frr_batch_run(exps, precision="f32")
    assert stats["status"] == 0
    for e, (w, r) in enumerate(zip(wls, res)):
        W = np.stack([O.assignment(w.philox_seed, int(k), w.n, w.n1) for k in r["keys"]])
        want = O.randtest(W, W[0], Ys[e], w.tau_grid, 0.05)
        mismatch = r["count"] != want["count"]
        assert np.all(want["near_ties"][mismatch] > 0) and mismatch.sum() <= 2
        assert r["ci_lo"] == want["ci_lo"] and r["ci_hi"] == want["ci_hi"]


def test_two_shards_on_one_gpu_merge_to_the_single_pool():
    from paper_2501_07642_b300.distributed import global_k, merge_accepted, shard, shard_q
    X = ar1_covariates(200, 100, 77, 0.5)
    B, q, seed = 100_000, 0.01, 21
    K = global_k(q, B)
    with frr.Context(X, 100, precision="split_bf16", whiten="chol") as ctx:
        want = frr.frr_select(ctx, seed, 500, B, q=q)
        parts = []
        for r in range(2):
            off, cnt = shard(B, r, 2)
            parts.append(frr.frr_select(ctx, seed, 500 + off, cnt, q=shard_q(K, cnt)))
    keys, m = merge_accepted(parts, K)
    assert np.array_equal(keys, want[0]) and np.array_equal(m, want[1])


def test_batch_paths_agree_with_single_calls():
    """One batch mixing the driver's paths -- q mode with host buffers (chains enqueued
    without read-backs), q mode with device outputs (keys placed directly), q mode with
    device test inputs and threshold mode (both one by one) -- against frr_select +
    frr_randtest on single contexts."""
    import ctypes
    import torch

    dev = torch.device("cuda")
    specs = [("host", 0.01), ("dev_out", 0.01), ("dev_in", 0.02), ("thr", None)]
    exps = (frr.frr_experiment * len(specs))()
    keep, want = [], []
    for k, (kind, q) in enumerate(specs):
        n, d = (120 + 40 * k, 30 + 11 * k)
        X = ar1_covariates(n, d, 900 + k, 0.3)
        Y = np.ascontiguousarray(X[:, 0] + np.random.default_rng(k).standard_normal(n))
        tau = np.linspace(-1.0, 1.0, 41)
        seed, first, B = 50 + k, 1000 * k, 12_000
        with frr.Context(X, n // 2, precision="split_bf16", whiten="chol") as ctx:
            if q is None:
                ref_keys, ref_m = frr.frr_select(ctx, seed, first, B, q=0.004)
                thr = float(ref_m.max())
                sk, sm = frr.frr_select(ctx, seed, first, B, threshold=thr)
            else:
                thr = math.nan
                sk, sm = frr.frr_select(ctx, seed, first, B, q=q)
            rt = frr.frr_randtest(ctx, seed, sk, int(sk[0]), Y, tau)
            p, cnt, lo, hi = rt["p"], rt["count"], rt["ci_lo"], rt["ci_hi"]
        want.append((sk, sm, p, cnt, lo, hi))
        a = exps[k]
        a.X = X.ctypes.data
        a.n, a.d, a.n1 = n, d, n // 2
        a.whiten = frr.WHITEN["chol"]
        a.ridge = 0.1
        a.seed, a.first_draw, a.B = seed, first, B
        a.q = math.nan if q is None else q
        a.threshold = thr
        cap = 4096
        a.cap = cap
        a.T = tau.size
        a.alpha = 0.05
        if kind == "dev_out":
            bufs = dict(keys=torch.zeros(cap, dtype=torch.int64, device=dev), m=torch.zeros(cap, dtype=torch.float64, device=dev),
                        p=torch.zeros(tau.size, dtype=torch.float64, device=dev),
                        c=torch.zeros(tau.size, dtype=torch.int64, device=dev))
            a.keys_out, a.M64_out = bufs["keys"].data_ptr(), bufs["m"].data_ptr()
            a.p_out, a.count_out = bufs["p"].data_ptr(), bufs["c"].data_ptr()
            a.Y, a.tau = Y.ctypes.data, tau.ctypes.data
        else:
            bufs = dict(keys=np.zeros(cap, dtype=np.uint64), m=np.zeros(cap), p=np.zeros(tau.size),
                        c=np.zeros(tau.size, dtype=np.int64))
            a.keys_out, a.M64_out = bufs["keys"].ctypes.data, bufs["m"].ctypes.data
            a.p_out, a.count_out = bufs["p"].ctypes.data, bufs["c"].ctypes.data
            if kind == "dev_in":
                bufs["Yd"] = torch.from_numpy(Y).to(dev)
                bufs["td"] = torch.from_numpy(tau).to(dev)
                a.Y, a.tau = bufs["Yd"].data_ptr(), bufs["td"].data_ptr()
            else:
                a.Y, a.tau = Y.ctypes.data, tau.ctypes.data
        keep += [X, Y, tau, bufs]
    st = frr.frr_batch_stats()
    opts = frr.frr_default_opts()
    rc = frr.lib().frr_batch_run(ctypes.addressof(exps), len(specs), ctypes.byref(opts), ctypes.byref(st))
    torch.cuda.synchronize()
    assert rc == 0, [exps[k].status for k in range(len(specs))]
    for k, (kind, q) in enumerate(specs):
        sk, sm, p, cnt, lo, hi = want[k]
        a, bufs = exps[k], keep[4 * k + 3]
        K = a.K_out
        assert a.status == 0 and K == len(sk), kind
        get = (lambda t: t.cpu().numpy()) if kind == "dev_out" else (lambda t: t)
        assert np.array_equal(get(bufs["keys"])[:K].astype(np.uint64), sk), kind
        assert np.array_equal(get(bufs["m"])[:K], sm), kind
        assert np.array_equal(get(bufs["p"]), p) and np.array_equal(get(bufs["c"]), cnt), kind
        same = lambda u, v: u == v or (math.isnan(u) and math.isnan(v))
        assert same(a.ci_lo, lo) and same(a.ci_hi, hi), kind


@pytest.mark.parametrize("path", ["select", "batch"])
def test_heavily_tied_pool_overflows_the_deferred_buffer_and_is_redone(path):
    """One binary covariate: M takes a handful of values, so about a quarter of the draws tie
    at the smallest M and the retained set (far more than 4 K + 16384 draws) outgrows the
    buffer of a deferred selection. The selection is redone without deferral and must still
    return the K draws with the smallest (M, index), as the oracle does."""
    n, B, q, seed = 40, 200_000, 0.001, 33
    X = np.zeros((n, 1))
    X[: n // 2, 0] = 1.0
    if path == "select":
        with frr.Context(X, n // 2, whiten="diag") as ctx:
            keys, m64 = frr.frr_select(ctx, seed, 0, B, q=q)
    else:
        res, st = frr.frr_batch_run([dict(X=X, n1=n // 2, whiten="diag", seed=seed, B=B, q=q)])
        assert st["status"] == 0
        keys, m64 = res[0]["keys"], res[0]["m64"]
    Zc, *_ = O.prep(X, "diag", 0.0)
    M = O.balance(Zc, n // 2, seed, 0, B)
    wk, wm = O.select_from_M(M, 0, q=q)
    assert np.sum(M <= wm.max()) > 4 * len(wk) + 16384  # the overflow really happens
    assert np.array_equal(keys, wk)
    assert np.allclose(m64, wm, rtol=1e-11, atol=1e-300)
