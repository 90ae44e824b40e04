"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

None of these tests re-types an oracle formula: each compares the oracle with
a published value, a closed form, an invariant, a library routine, or brute
force, so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them.
"""
import itertools
import math
from pathlib import Path

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

GOLDEN = Path(__file__).resolve().parent / "golden"


def _gauss(n, d, seed):
    return np.random.default_rng(seed).standard_normal((n, d))


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answer_vectors(oracle):
    rows = [l.split() for l in (GOLDEN / "philox4x32_10_kat.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_unit_word_counter_layout(oracle):
    # unit i reads word i mod 4 of the block with counter (i // 4, 0, lo(b), hi(b)),
    # key (lo(seed), hi(seed))
    seed, draw, n = 0x1234_5678_9ABC_DEF0, (7 << 32) + 11, 13
    words = oracle.unit_words(seed, draw, n)
    for i in range(n):
        blk = oracle.philox4x32_10([i // 4, 0, draw & 0xFFFFFFFF, draw >> 32],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        assert words[i] == blk[i % 4]


# ------------------------------------------------------------ assignment ----
@pytest.mark.parametrize("n,n1", [(2, 1), (3, 1), (3, 2), (20, 10), (33, 5), (100, 50), (129, 64), (1000, 500)])
def test_assignment_has_exactly_n1_treated(oracle, n, n1):
    W = oracle.assignments(seed=99, first=5, count=40, n=n, n1=n1)
    assert W.shape == (40, n)
    assert set(np.unique(W)) <= {0, 1}
    assert np.all(W.sum(axis=1) == n1)


def test_assignment_is_smallest_pairs_by_library_sort(oracle):
    n, n1 = 57, 20
    for draw in range(25):
        r = oracle.unit_words(4242, draw, n).astype(np.int64)
        order = np.lexsort((np.arange(n), r))  # primary key r, then unit index
        ref = np.zeros(n, dtype=np.uint8)
        ref[order[:n1]] = 1
        assert np.array_equal(ref, oracle.assignment(4242, draw, n, n1))


def test_assignment_uniform_over_all_subsets(oracle):
    # complete randomization: every one of the C(6,3) = 20 subsets equally likely
    n, n1, B = 6, 3, 200_000
    W = oracle.assignments(seed=1, first=0, count=B, n=n, n1=n1)
    codes = (W.astype(np.int64) << np.arange(n)).sum(axis=1)
    subsets = [sum(1 << i for i in c) for c in itertools.combinations(range(n), n1)]
    counts = np.array([(codes == s).sum() for s in subsets])
    assert counts.sum() == B
    chi2 = ((counts - B / 20) ** 2 / (B / 20)).sum()
    assert scipy.stats.chi2.sf(chi2, 19) > 1e-4
    # marginal and pairwise inclusion probabilities
    marg = W.mean(axis=0)
    assert np.all(np.abs(marg - n1 / n) < 5 * math.sqrt(0.25 / B))
    pair = (W[:, 0] & W[:, 1]).mean()
    assert abs(pair - n1 * (n1 - 1) / (n * (n - 1))) < 5 * math.sqrt(0.25 / B)


# ----------------------------------------------------------- enumeration ----
@pytest.mark.parametrize("n,n1", [(1, 1), (5, 2), (10, 5), (12, 4), (20, 10)])
def test_enumeration_visits_every_subset_once_in_increasing_order(oracle, n, n1):
    masks = oracle.enum_masks(n, n1)
    assert masks.size == math.comb(n, n1)
    ref = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), n1))
    assert [int(m) for m in masks] == ref
    # a window starting at a rank is the same slice
    if masks.size > 10:
        assert np.array_equal(oracle.enum_masks(n, n1, first=7, count=3), masks[7:10])


@pytest.mark.parametrize("n,n1", [(1, 1), (10, 1), (10, 9), (12, 3), (16, 8)])
def test_rank_and_unrank_follow_the_enumeration_order(oracle, n, n1):
    # the brute-force order (sorted integer masks) fixes every rank
    ref = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), n1))
    assert [oracle.mask_of_rank(n, n1, r) for r in range(len(ref))] == ref
    assert [oracle.rank_of_mask(m) for m in ref] == list(range(len(ref)))


def test_unrank_at_the_largest_supported_n(oracle):
    n, n1 = 63, 31
    N = math.comb(n, n1)
    assert oracle.mask_of_rank(n, n1, 0) == (1 << n1) - 1
    assert oracle.mask_of_rank(n, n1, N - 1) == ((1 << n) - 1) ^ ((1 << (n - n1)) - 1)
    rng = np.random.default_rng(3)
    for r in rng.integers(0, N, size=200, dtype=np.uint64):
        m = oracle.mask_of_rank(n, n1, int(r))
        assert bin(m).count("1") == n1 and m < (1 << n)
        assert oracle.rank_of_mask(m) == int(r)


@pytest.mark.parametrize("n", [10, 16])
def test_complement_reverses_the_rank_when_groups_are_equal(oracle, n):
    # with n1 = n / 2 the complement of rank r sits at rank C(n, n1) - 1 - r (brute force)
    n1 = n // 2
    masks = oracle.enum_masks(n, n1)
    full = (1 << n) - 1
    N = masks.size
    assert all(oracle.rank_of_mask(full ^ int(masks[r])) == N - 1 - r for r in range(N))


# ----------------------------------------------------------------- prep ----
@pytest.mark.parametrize("whiten,ridge", [("chol", 0.0), ("ridge", 0.1), ("diag", 0.0)])
def test_prep_against_library_routines(oracle, whiten, ridge):
    n, d = 40, 7
    X = _gauss(n, d, 3) @ np.random.default_rng(4).standard_normal((d, d)) + 2.5
    Zc, L, xbar, S = oracle.prep(X, whiten, ridge)
    assert np.allclose(xbar, X.mean(axis=0), rtol=1e-14, atol=1e-14)
    assert np.allclose(S, np.cov(X, rowvar=False, ddof=1), rtol=1e-12, atol=1e-13)
    if whiten == "diag":
        Lref = np.diag(np.sqrt(np.diag(S)))
    else:
        Sl = S + ridge * np.trace(S) / d * np.eye(d)
        Lref = np.linalg.cholesky(Sl)
    assert np.allclose(L, Lref, rtol=1e-12, atol=1e-13)
    Zref = scipy.linalg.solve_triangular(Lref, (X - X.mean(axis=0)).T, lower=True).T
    assert np.allclose(Zc, Zref, rtol=1e-11, atol=1e-12)
    if whiten == "chol":
        assert np.allclose(Zc.T @ Zc / (n - 1), np.eye(d), atol=1e-12)
    assert np.allclose(Zc.sum(axis=0), 0.0, atol=1e-11)


def test_prep_rejects_singular_covariance(oracle):
    X = _gauss(6, 8, 5)  # d > n - 1: rank-deficient S
    with pytest.raises(ValueError):
        oracle.prep(X, "chol")
    Zc, *_ = oracle.prep(X, "ridge", 0.1)  # the ridge makes it definite
    assert np.isfinite(Zc).all()


# -------------------------------------------------------------- balance ----
def _all_assignments(n, n1):
    for c in itertools.combinations(range(n), n1):
        w = np.zeros(n, dtype=np.uint8)
        w[list(c)] = 1
        yield w


@pytest.mark.parametrize("n,n1,d", [(10, 5, 3), (12, 5, 4), (9, 2, 1)])
def test_mean_of_M_over_all_assignments_is_d(oracle, n, n1, d):
    # Under complete randomization with n-1 covariance denominators,
    # (n1 n0 / n) E[Delta Delta^T] = S, so E[T^2] = tr(S^{-1} S) = d exactly.
    X = _gauss(n, d, 10 + n)
    Zc, *_ = oracle.prep(X, "chol")
    Ms = [oracle.M_of(Zc, w) for w in _all_assignments(n, n1)]
    assert abs(np.mean(Ms) - d) < 1e-12 * d


def test_mean_of_M_ridge_and_diag_closed_forms(oracle):
    n, n1, d = 11, 5, 4
    X = _gauss(n, d, 21) @ np.array([[1, .5, 0, 0], [0, 1, .3, 0], [0, 0, 1, .8], [0, 0, 0, 1.]])
    S = np.cov(X, rowvar=False, ddof=1)
    Zr, *_ = oracle.prep(X, "ridge", 0.1)
    Sl = S + 0.1 * np.trace(S) / d * np.eye(d)
    want = np.trace(np.linalg.solve(Sl, S))
    Ms = [oracle.M_of(Zr, w) for w in _all_assignments(n, n1)]
    assert abs(np.mean(Ms) - want) < 1e-12 * want
    Zd, *_ = oracle.prep(X, "diag")
    Md = [oracle.M_of(Zd, w) for w in _all_assignments(n, n1)]
    assert abs(np.mean(Md) - d) < 1e-12 * d


def test_M_affine_invariance_under_chol(oracle):
    n, d = 30, 6
    rng = np.random.default_rng(7)
    X = rng.standard_normal((n, d))
    A = rng.standard_normal((d, d)) + 3 * np.eye(d)
    b = rng.standard_normal(d) * 10
    Z1, *_ = oracle.prep(X, "chol")
    Z2, *_ = oracle.prep(X @ A + b, "chol")
    for draw in range(20):
        w = oracle.assignment(5, draw, n, 15)
        m1, m2 = oracle.M_of(Z1, w), oracle.M_of(Z2, w)
        assert abs(m1 - m2) <= 1e-10 * m1


def test_M_complement_symmetry_is_bit_exact(oracle):
    n, d = 24, 5
    Zc, *_ = oracle.prep(_gauss(n, d, 8), "chol")
    for draw in range(50):
        w = oracle.assignment(3, draw, n, n // 2)
        assert oracle.M_of(Zc, w) == oracle.M_of(Zc, 1 - w)


def test_M_d1_is_squared_standardised_mean_difference(oracle):
    # Sec. 2.2: M reduces to the squared SMD; in T^2 units times n1 n0 / n
    n, n1 = 15, 6
    x = np.random.default_rng(9).standard_normal((n, 1)) * 3 + 1
    Zc, *_ = oracle.prep(x, "chol")
    for draw in range(20):
        w = oracle.assignment(11, draw, n, n1).astype(bool)
        diff = x[w, 0].mean() - x[~w, 0].mean()
        want = n1 * (n - n1) / n * diff ** 2 / x[:, 0].var(ddof=1)
        assert abs(oracle.M_of(Zc, w.astype(np.uint8)) - want) <= 1e-12 * max(want, 1e-300) + 1e-15


def test_M_is_constant_when_d_is_n_minus_1(oracle):
    # Zc Zc^T = (n-1)(I - 11^T/n) when d = n-1, so every assignment has M = n-1
    n, d = 12, 11
    Zc, *_ = oracle.prep(_gauss(n, d, 12), "chol")
    Ms = [oracle.M_of(Zc, oracle.assignment(2, b, n, 6)) for b in range(30)]
    assert np.allclose(Ms, n - 1, rtol=1e-9)


def test_M_equals_scaled_squared_norm_of_treated_sum(oracle):
    # spec form: M = n/(n1 n0) * ||w^T Zc||^2 (equal because sum_i Zc_i = 0)
    n, n1, d = 50, 20, 9
    Zc, *_ = oracle.prep(_gauss(n, d, 13), "ridge", 0.05)
    W = oracle.assignments(17, 0, 30, n, n1)
    s = W.astype(np.float64) @ Zc
    want = n / (n1 * (n - n1)) * (s ** 2).sum(axis=1)
    got = oracle.balance(Zc, n1, 17, 0, 30)
    assert np.allclose(got, want, rtol=1e-11)


def test_balance_batch_matches_single_calls(oracle):
    n, n1, d = 20, 10, 5
    Zc, *_ = oracle.prep(_gauss(n, d, 0), "chol")
    got = oracle.balance(Zc, n1, None, 100, 50)  # exact ranks 100..149
    masks = oracle.enum_masks(n, n1, 100, 50)
    W = oracle.masks_to_w(masks, n)
    assert np.array_equal(got, [oracle.M_of(Zc, w) for w in W])
    got2 = oracle.balance_list(Zc, n1, 77, [3, 9, 1])
    assert np.array_equal(got2, [oracle.M_of(Zc, oracle.assignment(77, b, n, n1)) for b in (3, 9, 1)])


# ------------------------------------------------------------- selection ----
def test_accepted_counts_printed_in_paper(oracle):
    rows = [l.split() for l in (GOLDEN / "paper_acceptance_counts.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    for q, B, K, pmin in rows:
        k = oracle.k_from_q(float(q), int(float(B)))
        assert k == int(K)
        assert f"{1.0 / k:.4f}" == pmin


def test_selection_is_brute_force_best_q_fraction(oracle):
    n, n1, d, B, q = 30, 15, 4, 3000, 0.01
    Zc, *_ = oracle.prep(_gauss(n, d, 14), "chol")
    keys, M = oracle.select(Zc, n1, 123, 1000, B, q=q)
    assert keys.size == 30
    allM = oracle.balance(Zc, n1, 123, 1000, B)
    order = np.lexsort((np.arange(B), allM))
    want = np.sort(order[:30] + 1000)
    assert np.array_equal(keys, want)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    assert M.max() <= np.delete(allM, order[:30]).min()


def test_selection_ties_go_to_lower_index(oracle):
    # exact enumeration with n1 = n0: every M appears for a mask and its complement
    n, n1, d = 10, 5, 2
    Zc, *_ = oracle.prep(_gauss(n, d, 15), "chol")
    total = math.comb(n, n1)
    M = oracle.balance(Zc, n1, None, 0, total)
    keys, _ = oracle.select_from_M(M, 0, q=3 / total)  # K = 3: splits a tied pair
    order = sorted(range(total), key=lambda b: (M[b], b))
    assert list(keys) == sorted(order[:3])
    m3 = M[order[2]]
    tied = [b for b in range(total) if M[b] == m3]
    assert len(tied) == 2 and order[2] == min(tied)


def test_threshold_mode_keeps_all_at_or_below(oracle):
    n, n1, d = 12, 6, 3
    Zc, *_ = oracle.prep(_gauss(n, d, 16), "chol")
    total = math.comb(n, n1)
    M = oracle.balance(Zc, n1, None, 0, total)
    a = float(np.sort(M)[40])
    keys, Mk = oracle.select_from_M(M, 0, threshold=a)
    assert np.array_equal(keys, np.flatnonzero(M <= a))


# ------------------------------------------------------ randomization test ----
def _textbook_exact_p(y, w_obs, tau, n, n1):
    """Exact randomization p-value of the sharp null Y(1) = Y(0) + tau, two-sided
    difference in means over all C(n, n1) assignments (plain Python)."""
    y0 = [y[i] - tau * w_obs[i] for i in range(n)]

    def dim(w):
        t = sum(y0[i] for i in range(n) if w[i]) / n1
        c = sum(y0[i] for i in range(n) if not w[i]) / (n - n1)
        return t - c

    t_obs = abs(dim(w_obs))
    cnt = tot = 0
    for comb in itertools.combinations(range(n), n1):
        w = [0] * n
        for i in comb:
            w[i] = 1
        tot += 1
        cnt += abs(dim(w)) >= t_obs - 1e-12 * (t_obs + 1)
    return cnt / tot


def test_randtest_full_enumeration_is_textbook_exact_p(oracle):
    n, n1 = 10, 5
    rng = np.random.default_rng(31)
    W = oracle.masks_to_w(oracle.enum_masks(n, n1), n)
    w_obs = W[17]
    y = rng.standard_normal(n) + 0.8 * w_obs
    taus = np.array([-1.0, 0.0, 0.4, 1.5])
    res = oracle.randtest(W, w_obs, y, taus)
    for g, tau in enumerate(taus):
        assert res["p"][g] == pytest.approx(_textbook_exact_p(y, w_obs, tau, n, n1), abs=1e-15)
        assert res["count"][g] >= 1


def test_randtest_p_is_one_at_the_point_estimate_and_at_least_one_over_K(oracle):
    n, n1 = 40, 20
    W = oracle.assignments(8, 0, 500, n, n1)
    w_obs = W[0]
    rng = np.random.default_rng(2)
    y = rng.standard_normal(n) * 0.01 + 50.0 * w_obs  # w_obs is by far the most extreme
    a_obs = oracle.dim(y, w_obs)
    res = oracle.randtest(W, w_obs, y, np.array([0.0, a_obs]))
    assert res["count"][0] == 1 and res["p"][0] == pytest.approx(1 / 500)
    assert res["p"][1] >= 1 - 2 / 500  # |t_obs| is (numerically) zero at tau = DiM(Y)


def test_randtest_interval_is_grid_points_with_p_above_alpha(oracle):
    n, n1 = 30, 15
    W = oracle.assignments(9, 0, 400, n, n1)
    w_obs = W[0]
    y = np.random.default_rng(3).standard_normal(n) + 1.0 * w_obs
    grid = np.round(np.linspace(-2, 4, 121), 12)
    res = oracle.randtest(W, w_obs, y, grid, alpha=0.05)
    keep = grid[res["p"] > 0.05]
    assert res["ci_lo"] == keep.min() and res["ci_hi"] == keep.max()
    assert res["ci_lo"] <= oracle.dim(y, w_obs) <= res["ci_hi"]
    res2 = oracle.randtest(W, w_obs, y, np.array([100.0]), alpha=0.05)
    assert math.isnan(res2["ci_lo"]) and math.isnan(res2["ci_hi"])


# -------------------------------------------------------------- distances ----
def test_distance_matches_library_cdist(oracle):
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(21)
    X = rng.standard_normal((37, 19)).astype(np.float32)
    Y = (rng.standard_normal((23, 19)) * 3 + 1).astype(np.float32)
    want = cdist(X.astype(np.float64), Y.astype(np.float64))
    assert np.allclose(oracle.distance(X, Y), want, rtol=1e-13, atol=0)
    assert np.allclose(oracle.distance(X, Y, squared=True), want ** 2, rtol=1e-12, atol=0)


def test_distance_self_is_symmetric_with_zero_diagonal(oracle):
    X = np.random.default_rng(22).standard_normal((30, 7)).astype(np.float32)
    D = oracle.distance(X)
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0.0)


def test_distance_closed_forms(oracle):
    # points on two axes: |a e1 - b e2| = sqrt(a^2 + b^2); integer shifts leave distances unchanged
    X = np.zeros((3, 4), dtype=np.float32)
    Y = np.zeros((2, 4), dtype=np.float32)
    X[:, 0] = [3, 5, 8]
    Y[:, 1] = [4, 12]
    D = oracle.distance(X, Y)
    assert np.array_equal(D, np.sqrt(np.array([[9 + 16, 9 + 144], [25 + 16, 25 + 144], [64 + 16, 64 + 144]])))
    assert np.array_equal(oracle.distance(X + 7, Y + 7), D)


def test_distance_pairs_are_entries_of_the_matrix(oracle):
    rng = np.random.default_rng(23)
    X = rng.standard_normal((11, 5)).astype(np.float32)
    Y = rng.standard_normal((13, 5)).astype(np.float32)
    ij = np.stack([rng.integers(0, 11, 40), rng.integers(0, 13, 40)], axis=1)
    D = oracle.distance(X, Y)
    assert np.array_equal(oracle.distance_pairs(X, Y, ij), D[ij[:, 0], ij[:, 1]])
