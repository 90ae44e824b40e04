"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: assignments, key streams and accepted key sets bit-exact / identical;
M and test statistics within 1e-5 relative of FP64; exact p-value counts
(grid points whose comparison is a numerical near-tie on either side are
excluded from the count check and must be rare).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import (ar1_covariates, mixed_standardised_covariates, outcome, workload)

pytestmark = pytest.mark.gpu

REL_M = 1e-5          # approximate M (bulk path) vs FP64


def _m_err(got, want, precision, d):
    """Error of the approximate M. FP32: relative to M. Split BF16 (two 8-bit-significand
    parts, ~2^-17 relative per covariate entry): relative to the scale of the statistic,
    max(M, d) with E[M] = d under Cholesky whitening, because near M = 0 the absolute error
    (about 1e-6 here) dominates a relative measure."""
    scale = want if precision == "f32" else np.maximum(want, d)
    return (np.abs(got - want) / scale).max()
REL_M64 = 1e-11       # exact-sum recheck vs the oracle's FP64 M
# Whitened covariates from the tensor-core covariance vs the oracle's FP64 chain, relative to
# each column's largest |Zc|: both covariances are within about n 2^-53 max|Xc_.j| max|Xc_.k|
# of the exact one, and the whitening multiplies that by the conditioning of S (tens here),
# so agreement is expected near 1e-15; the bar leaves four orders of magnitude.
REL_ZC_TC = 1e-11
PRECISIONS = ["f32", "split_bf16"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_07642_b300 import build
    build.build_library()
    O.build()


def _ctx(X, n1, precision="f32", whiten="chol", ridge=0.1, prep="tensor"):
    return frr.Context(X, n1, precision=precision, whiten=whiten, ridge=ridge, prep=prep)


# ------------------------------------------------------------ assignments ----
@pytest.mark.parametrize("n,n1", [(2, 1), (3, 2), (5, 2), (20, 10), (31, 7), (64, 32), (100, 50), (127, 1),
                                  (128, 127), (129, 64), (255, 100), (256, 128), (500, 250), (1000, 500),
                                  (1024, 512), (2000, 1000), (2048, 1)])
def test_assignments_bit_exact(n, n1):
    X = ar1_covariates(n, 1, 5, 0.0)
    seed, first, count = 0xDEADBEEF12345678, (3 << 32) + 17, 300
    with _ctx(X, n1, whiten="diag") as ctx:
        got = frr.frr_assignments(ctx, seed, first, count)
        single = frr.frr_assignment(ctx, seed, first + 7)
    want = O.assignments(seed, first, count, n, n1)
    assert np.array_equal(got, want)
    assert np.array_equal(single, want[7])


def test_assignments_first_10k_draws_n1000():
    n, n1 = 1000, 500
    X = ar1_covariates(n, 2, 6, 0.0)
    with _ctx(X, n1, whiten="diag") as ctx:
        got = frr.frr_assignments(ctx, 3, 0, 10_000)
    assert np.array_equal(got, O.assignments(3, 0, 10_000, n, n1))


def test_exact_enumeration_all_ranks_n20():
    n, n1 = 20, 10
    X = ar1_covariates(n, 5, 0, 0.0)
    with _ctx(X, n1) as ctx:
        got = frr.frr_assignments(ctx, frr.FRR_EXACT_SEED, 0, 184_756)
    want = O.masks_to_w(O.enum_masks(n, n1), n)
    assert np.array_equal(got, want)


# --------------------------------------------------------------- whitening ----
@pytest.mark.parametrize("n,d,whiten", [(60, 10, "chol"), (100, 100, "ridge"), (40, 7, "diag"), (333, 129, "chol")])
def test_whitened_covariates_bit_exact(n, d, whiten):
    X = ar1_covariates(n, d, 40 + d, 0.5) * 3.0 + 1.5
    with _ctx(X, n // 2, whiten=whiten, prep="fp64_chain") as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, whiten, 0.1)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("case", ["wide_scales", "zero_column", "tiny_and_huge", "all_tiny", "subnormal_cov"])
def test_whitened_covariates_bit_exact_extreme_magnitudes(case):
    """Bit patterns (signed zeros included) at magnitudes that reach the divisions' safe-range
    edges: columns scaled by powers of two far from 1, an exactly constant column whose
    whitened entries are exact zeros, and covariates so small (2^-500) that the covariances
    (~2^-1000) and pivots (~2^-500) fall outside the fast division's exponent range."""
    n, d = 90, 40
    X = ar1_covariates(n, d, 77, 0.4)
    if case == "wide_scales":
        X = X * np.exp2(np.linspace(-240, 240, d))[None, :]
    elif case == "zero_column":
        X[:, 3] = 2.5
        X[:, 17] = 0.0
    elif case == "tiny_and_huge":
        X[:, : d // 2] *= 2.0 ** -300
        X[:, d // 2:] *= 2.0 ** 300
    elif case == "subnormal_cov":
        X = X * 2.0 ** -515  # covariances and pivots near 2^-1030: subnormal
    else:
        X = X * 2.0 ** -500
    with _ctx(X, n // 2, whiten="ridge", prep="fp64_chain") as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, "ridge", 0.1)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_whitened_precision_workload_bit_exact():
    w = workload("precision_n1000_d1000")
    X = w.covariates()
    with _ctx(X, w.n1, whiten="ridge", prep="fp64_chain") as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, "ridge", 0.1)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def _zc_err(got, want):
    scale = np.abs(want).max(axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    return (np.abs(got - want) / scale).max()


def _zc_tol(X, whiten, ridge=0.1):
    """REL_ZC_TC, or for an ill-conditioned covariance (d close to n - 1 under Cholesky
    whitening) 1e-14 cond(S_lambda): two FP64-accurate whitenings differ by up to about
    cond(S) u in each column's scale (1e-14 = 45 u). S_lambda from numpy, not the oracle."""
    if whiten == "diag":
        return REL_ZC_TC
    Xc = X - X.mean(axis=0)
    S = Xc.T @ Xc / (X.shape[0] - 1)
    if whiten == "ridge":
        S = S + ridge * np.trace(S) / S.shape[0] * np.eye(S.shape[0])
    return max(REL_ZC_TC, 1e-14 * np.linalg.cond(S))


@pytest.mark.parametrize("n,d,whiten,kind", [(60, 10, "chol", "ar1"), (100, 100, "ridge", "ar1"),
                                             (40, 7, "diag", "ar1"), (333, 129, "chol", "ar1"),
                                             (65, 257, "ridge", "ar1"), (2048, 300, "chol", "mixed"),
                                             (1000, 1000, "ridge", "mixed")])
def test_whitened_covariates_tensor_covariance(n, d, whiten, kind):
    """The default covariance (digit products summed exactly on the tensor cores, rounded once)
    against the oracle's FP64 chain: ragged tiles (d = 7, 129, 257, 300), one to four exact
    512-row blocks (n = 40 ... 2048), heavy-tailed columns (the mixed recipe's lognormal quarter)."""
    X = (ar1_covariates(n, d, 50 + d, 0.5) * 3.0 + 1.5 if kind == "ar1"
         else mixed_standardised_covariates(n, d, 60 + d))
    with _ctx(X, n // 2, whiten=whiten) as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, whiten, 0.1)
    assert _zc_err(got, want) < REL_ZC_TC


@pytest.mark.parametrize("n,d,whiten", [(3, 1, "chol"), (10, 1, "ridge"), (130, 128, "chol"), (300, 256, "chol"),
                                         (600, 512, "ridge"), (257, 255, "chol"), (64, 300, "diag")])
def test_whitened_tensor_mode_edge_shapes(n, d, whiten):
    """Tensor-core preparation at tile and block edges: one column, one or two exact 128-wide
    tiles, d = 256 (no forward-substitution block boundary), d = 512 (one boundary whose rest is
    a whole block), d = n - 2, and diagonal whitening with d > n."""
    X = ar1_covariates(n, d, 900 + d, 0.3) + 0.25
    with _ctx(X, n // 2, whiten=whiten) as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, whiten, 0.1)
    assert _zc_err(got, want) < _zc_tol(X, whiten)  # d = n - 2: cond(S) ~ 1e5-1e6


@pytest.mark.parametrize("prep", ["fp64_chain", "tensor"])
def test_whitened_repeated_shapes_replay_their_preparation(prep):
    """A single experiment's preparation is captured into a CUDA graph on the first call of its
    shape and replayed by later calls of that shape: every call must prepare its own covariates
    (new values, another ridge, another context's output arrays), also after its shape's
    graph was evicted by more shapes than are kept, and back again."""
    shapes = [(60, 20), (70, 33), (90, 40), (64, 64), (130, 100), (600, 300), (60, 20), (90, 40)]
    for rep in range(2):
        for i, (n, d) in enumerate(shapes):
            X = ar1_covariates(n, d, 1000 + 17 * i + rep, 0.3) + 0.5 * rep
            ridge = 0.1 if (i + rep) % 2 == 0 else 0.35
            with _ctx(X, n // 2, whiten="ridge", ridge=ridge, prep=prep) as ctx:
                got = frr.frr_whitened(ctx)
            want, *_ = O.prep(X, "ridge", ridge)
            if prep == "fp64_chain":
                assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (rep, n, d)
            else:
                assert _zc_err(got, want) < _zc_tol(X, "ridge", ridge), (rep, n, d)


def test_whitened_concurrent_preparations_of_one_shape():
    """Threads preparing experiments of one shape at the same time (the library call releases
    the interpreter lock): one captures or replays the shape's launch graph, the others find
    it in use and enqueue their launches themselves; each must get its own covariates'
    whitening (bit for bit with the FP64 chains)."""
    import threading
    n, d, T = 200, 150, 6
    Xs = [ar1_covariates(n, d, 3000 + i, 0.3) + 0.1 * i for i in range(T)]
    out, err = [None] * T, [None] * T

    def work(i):
        try:
            for _ in range(2):
                with _ctx(Xs[i], n // 2, whiten="ridge", prep="fp64_chain") as ctx:
                    out[i] = frr.frr_whitened(ctx)
        except Exception as e:  # reported below, on the test's thread
            err[i] = e

    threads = [threading.Thread(target=work, args=(i,)) for i in range(T)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in range(T):
        assert err[i] is None, err[i]
        want, *_ = O.prep(Xs[i], "ridge", 0.1)
        assert np.array_equal(out[i].view(np.uint64), want.view(np.uint64)), i


def test_whitened_at_the_largest_n():
    """n = 2048, the largest supported, with d = 600 (three 256-column blocks of the forward
    substitution, the last one partial; 19 panels): both preparation modes against one oracle
    run, bit for bit with the FP64 chains, within the derived tolerance with the tensor cores."""
    n, d = 2048, 600
    X = ar1_covariates(n, d, 2048, 0.3) * 1.5 - 0.25
    want, *_ = O.prep(X, "ridge", 0.1)
    with _ctx(X, n // 2, whiten="ridge", prep="fp64_chain") as ctx:
        got = frr.frr_whitened(ctx)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    with _ctx(X, n // 2, whiten="ridge", prep="tensor") as ctx:
        got = frr.frr_whitened(ctx)
    assert _zc_err(got, want) < _zc_tol(X, "ridge")


@pytest.mark.parametrize("prep", ["fp64_chain", "tensor"])
def test_non_finite_covariates_found_on_the_device(prep):
    """frr_init finds a non-finite covariate where the device centres X (no host scan when the
    preparation runs): NaN, +inf or -inf at the first, a middle or the last entry gives
    FRR_E_ARG, also when the shape's preparation is replayed from its graph, and a finite X of
    the same shape is prepared correctly afterwards."""
    n, d = 120, 40
    X = ar1_covariates(n, d, 4242, 0.3)
    for bad in (math.nan, math.inf, -math.inf):
        for at in ((0, 0), (n // 2, d // 3), (n - 1, d - 1)):
            Xb = X.copy()
            Xb[at] = bad
            with pytest.raises(frr.FrrError) as e:
                _ctx(Xb, n // 2, whiten="ridge", prep=prep)
            assert e.value.status == -1, (bad, at)
        with _ctx(X, n // 2, whiten="ridge", prep=prep) as ctx:
            got = frr.frr_whitened(ctx)
        want, *_ = O.prep(X, "ridge", 0.1)
        if prep == "fp64_chain":
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        else:
            assert _zc_err(got, want) < _zc_tol(X, "ridge")


@pytest.mark.parametrize("case", ["wide_scales", "zero_column", "tiny_and_huge", "all_tiny", "subnormal_cov"])
def test_whitened_tensor_covariance_extreme_magnitudes(case):
    """Per-column power-of-two scales far from 1 (each column's digits are relative to its own
    largest entry), constant columns (centred to exact zeros: their whitened entries stay exact
    zeros), covariates at 2^-500 (products near 2^-1000, still normal) and at 2^-515 (subnormal
    covariances and pivots)."""
    n, d = 90, 40
    X = ar1_covariates(n, d, 77, 0.4)
    if case == "wide_scales":
        X = X * np.exp2(np.linspace(-240, 240, d))[None, :]
    elif case == "zero_column":
        X[:, 3] = 2.5
        X[:, 17] = 0.0
    elif case == "tiny_and_huge":
        X[:, : d // 2] *= 2.0 ** -300
        X[:, d // 2:] *= 2.0 ** 300
    elif case == "subnormal_cov":
        X = X * 2.0 ** -515  # covariances and pivots near 2^-1030: subnormal
    else:
        X = X * 2.0 ** -500
    with _ctx(X, n // 2, whiten="ridge") as ctx:
        got = frr.frr_whitened(ctx)
    want, *_ = O.prep(X, "ridge", 0.1)
    assert _zc_err(got, want) < REL_ZC_TC
    if case == "zero_column":
        assert np.all(got[:, [3, 17]] == 0.0)


# ---------------------------------------------------------------- balance ----
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n,d,whiten", [(100, 100, "ridge"), (20, 5, "chol"), (257, 33, "chol"), (1000, 1000, "ridge")])
def test_balance_within_1e5_of_fp64(precision, n, d, whiten):
    X = ar1_covariates(n, d, 7, 0.5)
    B = 2000 if n >= 1000 else 6000
    seed, first = 11, 123_456
    with _ctx(X, n // 2, precision, whiten) as ctx:
        got = frr.frr_balance(ctx, seed, first, B).astype(np.float64)
    Zc, *_ = O.prep(X, whiten, 0.1)
    want = O.balance(Zc, n // 2, seed, first, B)
    err = _m_err(got, want, precision, d)
    assert err < REL_M, err


@pytest.mark.parametrize("precision", PRECISIONS)
def test_balance_exact_ranks(precision):
    n, n1, d = 20, 10, 5
    X = ar1_covariates(n, d, 0, 0.0)
    with _ctx(X, n1, precision) as ctx:
        got = frr.frr_balance_exact(ctx, 1000, 5000).astype(np.float64)
    Zc, *_ = O.prep(X, "chol")
    want = O.balance(Zc, n1, None, 1000, 5000)
    assert _m_err(got, want, precision, d) < REL_M


def test_balance_to_device_buffer_matches_host_buffer():
    import torch
    X = ar1_covariates(100, 40, 8, 0.3)
    with _ctx(X, 50) as ctx:
        host = frr.frr_balance(ctx, 5, 0, 3000)
        dev = torch.empty(3000, dtype=torch.float32, device="cuda")
        frr.frr_balance(ctx, 5, 0, 3000, dev)
        torch.cuda.synchronize()
        assert np.array_equal(host, dev.cpu().numpy())


# ---------------------------------------------------------------- recheck ----
@pytest.mark.parametrize("n,d", [(1000, 300), (200, 64)])
def test_balance_independent_of_the_launch_range(n, d):
    """A draw's M_hat (Sec. 2.2, 2.3) depends only on its key: computed inside any range of
    draws -- one draw, fewer than a tile, a CTA count's worth of tiles plus one, an offset
    start -- it is bit for bit the value the launch over [0, 40000) gives. This covers how a
    launch splits its draws over CTAs and tiles (contiguous per-CTA ranges, the remainder in a
    CTA's first tile; CTAs with empty ranges)."""
    import torch
    X = ar1_covariates(n, d, 17, 0.4)
    with _ctx(X, n // 2, "split_bf16", "ridge") as ctx:
        ref = frr.frr_balance(ctx, 5, 0, 40_000)
        for first, B in [(0, 1), (5, 127), (1000, 129), (123, 148 * 128 + 1), (7, 20_000), (39_000, 1000),
                         (2, 148 * 72), (0, 40_000)]:
            got = torch.empty(B, dtype=torch.float32, device="cuda")
            frr.frr_balance(ctx, 5, first, B, got)
            torch.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy().view(np.uint32), ref[first:first + B].view(np.uint32)), (first, B)


@pytest.mark.parametrize("n,d,whiten", [(100, 100, "ridge"), (1000, 1000, "ridge"), (64, 20, "chol")])
def test_recheck_matches_oracle(n, d, whiten):
    X = ar1_covariates(n, d, 9, 0.5)
    draws = np.random.default_rng(1).integers(0, 1 << 40, 64).astype(np.uint64)
    with _ctx(X, n // 2, whiten=whiten) as ctx:
        got = frr.frr_recheck(ctx, 21, draws)
    Zc, *_ = O.prep(X, whiten, 0.1)
    want = O.balance_list(Zc, n // 2, 21, draws)
    assert np.allclose(got, want, rtol=REL_M64, atol=0)


def test_recheck_complement_pairs_bit_identical():
    n, n1, d = 20, 10, 5
    X = ar1_covariates(n, d, 0, 0.0)
    masks = O.enum_masks(n, n1)
    rank_of = {int(m): r for r, m in enumerate(masks)}
    full = (1 << n) - 1
    ranks = np.arange(0, 184_756, 997, dtype=np.uint64)
    comps = np.array([rank_of[full ^ int(masks[r])] for r in ranks], dtype=np.uint64)
    with _ctx(X, n1) as ctx:
        a = frr.frr_recheck(ctx, frr.FRR_EXACT_SEED, ranks)
        b = frr.frr_recheck(ctx, frr.FRR_EXACT_SEED, comps)
    assert np.array_equal(a, b)


# -------------------------------------------------------------- selection ----
def _oracle_select(X, n1, whiten, seed, first, B, q=None, threshold=None, threads=0):
    Zc, *_ = O.prep(X, whiten, 0.1)
    M = O.balance(Zc, n1, seed, first, B, threads=threads)
    return O.select_from_M(M, first, q=q, threshold=threshold) + (M,)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_select_exact_enumeration_workload(precision):
    w = workload("exact_n20_d5")
    X = w.covariates()
    total = math.comb(w.n, w.n1)
    with _ctx(X, w.n1, precision) as ctx:
        keys, m64 = frr.frr_select(ctx, frr.FRR_EXACT_SEED, 0, total, q=w.q)
        st = frr.frr_last_stats(ctx)
    wk, wm, _ = _oracle_select(X, w.n1, "chol", None, 0, total, q=w.q)
    assert len(keys) == 9238 == len(wk)
    assert np.array_equal(keys, wk)
    assert np.allclose(m64, wm, rtol=REL_M64, atol=0)
    assert st["band_violations"] == 0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_select_monte_carlo_workload(precision):
    w = workload("mc_n100_d100")
    X = w.covariates()
    with _ctx(X, w.n1, precision, w.whiten) as ctx:
        keys, m64 = frr.frr_select(ctx, w.philox_seed, 0, w.draws, q=w.q)
        st = frr.frr_last_stats(ctx)
    wk, wm, _ = _oracle_select(X, w.n1, w.whiten, w.philox_seed, 0, w.draws, q=w.q)
    assert len(keys) == 2000
    assert np.array_equal(keys, wk)
    assert np.allclose(m64, wm, rtol=REL_M64, atol=0)
    assert st["band_violations"] == 0 and st["max_err_over_band"] < 0.5
    assert st["max_rel_err"] < REL_M
    assert st["candidates"] >= 2000


def test_select_threshold_mode():
    """Threshold mode (Sec. 2.2 with a fixed acceptance threshold a) accepts the draws with
    M <= a. Against itself: a = the K-th accepted M64 of q mode gives the same draws. Against
    the oracle: a lies midway between two consecutive oracle M values, so the two sides agree
    however the last bits of M round (a threshold equal to some draw's M would not)."""
    w = workload("mc_n100_d100")
    X = w.covariates()
    B, K = 50_000, 500
    _, _, M = _oracle_select(X, w.n1, w.whiten, 1, 0, B, q=0.01)
    Ms = np.sort(M)
    assert Ms[K] - Ms[K - 1] > 1e-9 * Ms[K]
    a_mid = float(0.5 * (Ms[K - 1] + Ms[K]))
    with _ctx(X, w.n1, "f32", w.whiten) as ctx:
        k1, m1 = frr.frr_select(ctx, 1, 0, B, q=0.01)
        k2, m2 = frr.frr_select(ctx, 1, 0, B, threshold=float(np.max(m1)))
        k3, m3 = frr.frr_select(ctx, 1, 0, B, threshold=a_mid)
    assert len(k1) == K and np.array_equal(k1, k2)
    wk, wm = O.select_from_M(M, 0, threshold=a_mid)
    assert len(wk) == K
    assert np.array_equal(k3, wk)
    assert np.allclose(m3, wm, rtol=REL_M64, atol=0)


@pytest.mark.parametrize("mode", ["q", "threshold"])
def test_select_into_device_buffers_equals_host_buffers(mode):
    """Device outputs: in q mode the placement kernel writes the accepted keys straight into
    them (the count is K); in threshold mode they are copied after the read-back. Both must
    equal the host-buffer results, and a too-small device buffer must stay untouched."""
    import torch
    w = workload("mc_n100_d100")
    X = w.covariates()
    with _ctx(X, w.n1, "split_bf16", w.whiten) as ctx:
        hk, hm = frr.frr_select(ctx, 1, 500, 60_000, q=0.01)
        kw = dict(q=0.01) if mode == "q" else dict(threshold=float(hm.max()))
        hk, hm = frr.frr_select(ctx, 1, 500, 60_000, **kw)
        dk = torch.full((4096,), -1, dtype=torch.int64, device="cuda")
        dm = torch.full((4096,), -1.0, dtype=torch.float64, device="cuda")
        k, m = frr.frr_select(ctx, 1, 500, 60_000, keys_out=dk, M64_out=dm, cap=4096, **kw)
        K = len(hk)
        assert len(k) == K
        assert np.array_equal(dk[:K].cpu().numpy().astype(np.uint64), hk)
        assert np.array_equal(dm[:K].cpu().numpy(), hm)
        small = torch.full((K - 1,), -1, dtype=torch.int64, device="cuda")
        smallm = torch.full((K - 1,), -1.0, dtype=torch.float64, device="cuda")
        with pytest.raises(frr.FrrError) as e:
            frr.frr_select(ctx, 1, 500, 60_000, keys_out=small, M64_out=smallm, cap=K - 1, **kw)
        assert e.value.name == "FRR_E_CAPACITY"
        assert bool((small == -1).all()) and bool((smallm == -1.0).all())


def test_stream_in_shuffled_chunks_equals_one_select():
    w = workload("mc_n100_d100")
    X = w.covariates()
    with _ctx(X, w.n1, "f32", w.whiten) as ctx:
        k1, m1 = frr.frr_select(ctx, 1, 1000, 80_000, q=0.005)
        frr.frr_stream_begin(ctx, 1, 80_000, q=0.005)
        for first, cnt in [(61_000, 20_000), (1000, 30_000), (31_000, 30_000)]:
            frr.frr_stream_chunk(ctx, first, cnt)
        k2, m2 = frr.frr_stream_end(ctx, 1000)
    assert np.array_equal(k1, k2) and np.array_equal(m1, m2)


def test_select_capacity_and_state_errors():
    X = ar1_covariates(50, 5, 3, 0.0)
    with _ctx(X, 25) as ctx:
        with pytest.raises(frr.FrrError) as e:
            frr.frr_select(ctx, 1, 0, 10_000, q=0.01, cap=50)
        assert e.value.name == "FRR_E_CAPACITY"
        with pytest.raises(frr.FrrError) as e:
            frr.frr_stream_chunk(ctx, 0, 10)
        assert e.value.name == "FRR_E_STATE"
        with pytest.raises(frr.FrrError) as e:
            frr.frr_select(ctx, 1, (1 << 64) - 5, 10, q=0.5)
        assert e.value.name == "FRR_E_RANGE"
        with pytest.raises(frr.FrrError) as e:
            frr.frr_select(ctx, 1, 0, 10, q=0.5, threshold=1.0)
        assert e.value.name == "FRR_E_ARG"


@pytest.mark.parametrize("precision", PRECISIONS)
def test_select_n1000_d1000_identical_to_oracle(precision):
    X = mixed_standardised_covariates(1000, 1000, 103)
    B, q = 12_000, 0.01
    with _ctx(X, 500, precision, "ridge") as ctx:
        keys, m64 = frr.frr_select(ctx, 3, 0, B, q=q)
        st = frr.frr_last_stats(ctx)
    wk, wm, _ = _oracle_select(X, 500, "ridge", 3, 0, B, q=q)
    assert np.array_equal(keys, wk)
    assert np.allclose(m64, wm, rtol=REL_M64, atol=0)
    assert st["band_violations"] == 0 and st["max_rel_err"] < REL_M


@pytest.fixture(scope="module")
def precision_workload_oracle_pool():
    """The oracle's accepted pool of the whole precision workload (n = d = 1000, B = 2e5,
    q = 1e-3, K = 200): M in FP64 for every one of the 2e5 draws, then the K smallest
    (M, draw index). Also the relative gap between the K-th and (K+1)-th M."""
    w = workload("precision_n1000_d1000")
    X = w.covariates()
    Zc, *_ = O.prep(X, "ridge", 0.1)
    M = O.balance(Zc, w.n1, w.philox_seed, 0, w.draws)
    keys, m64 = O.select_from_M(M, 0, q=w.q)
    order = np.lexsort((np.arange(w.draws), M))
    gap = (M[order[len(keys)]] - M[order[len(keys) - 1]]) / M[order[len(keys) - 1]]
    return X, keys, m64, gap


@pytest.mark.parametrize("precision", PRECISIONS)
def test_select_precision_workload_full_size_identical_to_oracle(precision, precision_workload_oracle_pool):
    """Full precision workload, every draw scored by the oracle: the accepted key set is
    identical and M64 agrees to 1e-11 relative (Sec. 2.2, accept the best q fraction)."""
    X, wk, wm, gap = precision_workload_oracle_pool
    w = workload("precision_n1000_d1000")
    assert gap > 1e-11  # the K-th / (K+1)-th order does not rest on rounding
    with _ctx(X, w.n1, precision, "ridge") as ctx:
        keys, m64 = frr.frr_select(ctx, w.philox_seed, 0, w.draws, q=w.q)
        st = frr.frr_last_stats(ctx)
    assert len(keys) == 200 == len(wk)
    assert np.array_equal(keys, wk)
    assert np.allclose(m64, wm, rtol=REL_M64, atol=0)
    assert st["band_violations"] == 0 and st["max_rel_err"] < REL_M and st["parity_at_risk"] == 0


# ------------------------------------------------------- randomization test ----
def _check_counts(got, want):
    mismatch = got["count"] != want["count"]
    # a mismatch is allowed only at grid points where the oracle flags a near-tie
    assert np.all(want["near_ties"][mismatch] > 0)
    assert mismatch.sum() <= 2


def test_randtest_monte_carlo_workload():
    w = workload("mc_n100_d100")
    X = w.covariates()
    with _ctx(X, w.n1, "f32", w.whiten) as ctx:
        keys, _ = frr.frr_select(ctx, w.philox_seed, 0, w.draws, q=w.q)
        w_obs = frr.frr_assignment(ctx, w.philox_seed, int(keys[0]))
        Y = outcome(X, w_obs, w.tau_true, w.y_seed, w.noise_sd)
        got = frr.frr_randtest(ctx, w.philox_seed, keys, int(keys[0]), Y, w.tau_grid, 0.05)
    W = np.stack([O.assignment(w.philox_seed, int(k), w.n, w.n1) for k in keys])
    want = O.randtest(W, W[0], Y, w.tau_grid, 0.05)
    _check_counts(got, want)
    assert np.all(got["p"] >= 1.0 / len(keys))
    assert got["ci_lo"] == want["ci_lo"] and got["ci_hi"] == want["ci_hi"]
    assert np.allclose(got["p"], want["p"], atol=2.0 / len(keys))


def test_randtest_exact_workload():
    w = workload("exact_n20_d5")
    X = w.covariates()
    total = math.comb(w.n, w.n1)
    with _ctx(X, w.n1, "f32") as ctx:
        keys, _ = frr.frr_select(ctx, frr.FRR_EXACT_SEED, 0, total, q=w.q)
        w_obs = frr.frr_assignment(ctx, frr.FRR_EXACT_SEED, int(keys[0]))
        Y = outcome(X, w_obs, w.tau_true, w.y_seed, w.noise_sd)
        got = frr.frr_randtest(ctx, frr.FRR_EXACT_SEED, keys, int(keys[0]), Y, w.tau_grid, 0.05)
        with pytest.raises(frr.FrrError):
            frr.frr_randtest(ctx, frr.FRR_EXACT_SEED, keys[1:], int(keys[0]), Y, w.tau_grid, 0.05)
    W = O.masks_to_w(O.enum_masks(w.n, w.n1), w.n)[keys.astype(np.int64)]
    want = O.randtest(W, W[0], Y, w.tau_grid, 0.05)
    _check_counts(got, want)
    assert got["ci_lo"] == want["ci_lo"] and got["ci_hi"] == want["ci_hi"]


@pytest.mark.parametrize("n,n1", [(20, 10), (100, 50), (129, 1), (1000, 500), (2000, 1999), (2048, 1024)])
def test_warp_select_with_ties_matches_library_sort(n, n1):
    """Words with heavy ties (few distinct values) and ties exactly at the n1 boundary:
    the treated set is the n1 smallest (word, unit) pairs."""
    X = ar1_covariates(n, 1, 3, 0.0)
    rng = np.random.default_rng(n + n1)
    cases = [rng.integers(0, 4, n, dtype=np.uint64).astype(np.uint32),                 # 4 distinct values
             np.full(n, 0xffffffff, dtype=np.uint32),                                   # all equal, maximal
             rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)]
    w = cases[2].copy()
    srt = np.sort(w)
    w[w == srt[n1]] = srt[n1 - 1]                                                       # tie across the boundary
    cases.append(w)
    with _ctx(X, n1, whiten="diag") as ctx:
        for words in cases:
            got = frr.frr_assignment_from_words(ctx, words)
            order = np.lexsort((np.arange(n), words.astype(np.int64)))
            want = np.zeros(n, dtype=np.uint8)
            want[order[:n1]] = 1
            assert np.array_equal(got, want)
