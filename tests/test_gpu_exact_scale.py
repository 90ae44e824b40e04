"""Exact enumeration at scale (Sec. 2.3, randomization_type "exact"): every one of the
C(n, n1) assignments is balance-checked, streamed in chunks through the selection.

n = 28 (4.0e7 assignments): the oracle enumerates and scores all of them; the accepted
key sets must be identical. n = 36 (9.1e9 assignments): the oracle re-scores every
accepted rank and a seeded sample of ranks. With n1 = n0 an assignment and its
complement have the same M (exactly, on both sides), so the accepted set is closed under
complement except for the one pair that a cut of odd size splits, and there the lower
rank wins the tie. n = 63: ranks at the end of the C(63, 31) range.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr

pytestmark = pytest.mark.gpu

EXACT = (1 << 64) - 1   # FRR_EXACT_SEED
REL_M64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_07642_b300 import build
    build.build_library()
    O.build()


def _stream_all(ctx, N, q, chunk):
    frr.frr_stream_begin(ctx, EXACT, N, q=q)
    for first in range(0, N, chunk):
        frr.frr_stream_chunk(ctx, first, min(chunk, N - first))
    return frr.frr_stream_end(ctx, 1 << 14)


N28 = (28, 14, 5, 5e-5)


@pytest.fixture(scope="module")
def n28_oracle():
    n, n1, d, q = N28
    X = np.random.default_rng(28).standard_normal((n, d))
    Zc, *_ = O.prep(X, "chol")
    M = O.balance(Zc, n1, None, 0, math.comb(n, n1))
    keys, m = O.select_from_M(M, 0, q=q)
    return X, keys, m


@pytest.mark.parametrize("precision", ["split_bf16", "f32"])
def test_full_enumeration_n28_key_set_identical(precision, n28_oracle):
    n, n1, d, q = N28
    N = math.comb(n, n1)                      # 40,116,600
    X, want_keys, want_m = n28_oracle
    with frr.Context(X, n1, precision=precision, whiten="chol") as ctx:
        keys, m64 = _stream_all(ctx, N, q, 1 << 24)
        st = frr.frr_last_stats(ctx)
    assert st["band_violations"] == 0 and st["parity_at_risk"] == 0
    assert len(keys) == O.k_from_q(q, N)
    assert np.array_equal(keys, want_keys)
    assert np.allclose(m64, want_m, rtol=REL_M64, atol=0)


def test_enumeration_n36_9e9_assignments_complement_closed():
    n, n1, d = 36, 18, 8
    N = math.comb(n, n1)                      # 9,075,135,300
    q = 1.1e-7
    K = O.k_from_q(q, N)
    X = np.random.default_rng(36).standard_normal((n, d))
    with frr.Context(X, n1, precision="split_bf16", whiten="chol") as ctx:
        keys, m64 = _stream_all(ctx, N, q, 1 << 27)
        st = frr.frr_last_stats(ctx)
    assert st["band_violations"] == 0
    # an odd K splits a complement pair: an exact tie at the cut, which the statistics flag
    assert st["parity_at_risk"] == K % 2
    if K % 2:
        assert st["boundary_gap_rel"] == 0.0
    assert len(keys) == K
    ks = keys.astype(np.uint64)
    assert np.all(np.diff(ks.astype(np.int64)) > 0)
    Zc, *_ = O.prep(X, "chol")
    got = O.balance_list(Zc, n1, None, ks)
    assert np.allclose(m64, got, rtol=REL_M64, atol=0)
    # complement closure; the split pair (K odd) keeps its lower rank
    acc = set(int(k) for k in ks)
    unpaired = [k for k in acc if (N - 1 - k) not in acc]
    assert len(unpaired) == K % 2
    for k in unpaired:
        assert k < N - 1 - k
        assert O.balance_list(Zc, n1, None, np.array([N - 1 - k], dtype=np.uint64))[0] == \
            O.balance_list(Zc, n1, None, np.array([k], dtype=np.uint64))[0]
    # every sampled rejected rank comes after the last accepted one in (M, rank)
    kth = max(zip(got.tolist(), [int(k) for k in ks]))
    sample = np.random.default_rng(99).integers(0, N, size=200_000, dtype=np.uint64)
    sample = np.array([s for s in sample if int(s) not in acc], dtype=np.uint64)
    sm = O.balance_list(Zc, n1, None, sample)
    assert np.all((sm > kth[0]) | ((sm == kth[0]) & (sample.astype(np.int64) > kth[1])))


@pytest.mark.parametrize("precision", ["split_bf16", "f32"])
def test_exact_ranks_at_the_end_of_n63(precision):
    n, n1, d = 63, 31, 6
    N = math.comb(n, n1)
    X = np.random.default_rng(63).standard_normal((n, d))
    first = N - 5000
    with frr.Context(X, n1, precision=precision, whiten="chol") as ctx:
        got = frr.frr_balance_exact(ctx, first, 5000).astype(np.float64)
        with pytest.raises(frr.FrrError):
            frr.frr_balance_exact(ctx, N - 10, 11)
    Zc, *_ = O.prep(X, "chol")
    want = O.balance_list(Zc, n1, None, np.arange(first, N, dtype=np.uint64))
    scale = want if precision == "f32" else np.maximum(want, d)
    assert (np.abs(got - want) / scale).max() < 1e-5
