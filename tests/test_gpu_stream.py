"""Tight-threshold streaming workload: n = d = 1000, AR(1) rho = 0.5 covariates,
1e8 Philox draws streamed in 1e6-draw chunks, q = 1.2e-5 (K = 1200), split-BF16 bulk
path with the exact recheck. The oracle re-scores every accepted key and a seeded
sample of 1e5 draws; every sampled rejected draw must come after the last accepted one
in (M, draw index)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import workload

pytestmark = pytest.mark.gpu


def test_stream_1e8_draws_in_1e6_chunks():
    from paper_2501_07642_b300 import build
    build.build_library()
    w = workload("stream_n1000_d1000")
    X = w.covariates()
    with frr.Context(X, w.n1, precision="split_bf16", whiten=w.whiten, ridge=w.ridge) as ctx:
        frr.frr_stream_begin(ctx, w.philox_seed, w.draws, q=w.q)
        for first in range(0, w.draws, w.chunk):
            frr.frr_stream_chunk(ctx, first, w.chunk)
        keys, m64 = frr.frr_stream_end(ctx, 4096)
        st = frr.frr_last_stats(ctx)
    assert len(keys) == 1200
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    assert st["band_violations"] == 0 and st["parity_at_risk"] == 0
    Zc, *_ = O.prep(X, w.whiten, w.ridge)
    got = O.balance_list(Zc, w.n1, w.philox_seed, keys)
    assert np.allclose(m64, got, rtol=1e-11, atol=0)
    kth = max(zip(got, keys.tolist()))
    acc = set(keys.tolist())
    sample = np.random.default_rng(12345).choice(w.draws, 100_000, replace=False).astype(np.uint64)
    sample = np.array([s for s in sample if int(s) not in acc], dtype=np.uint64)
    sm = O.balance_list(Zc, w.n1, w.philox_seed, sample)
    assert np.all((sm > kth[0]) | ((sm == kth[0]) & (sample.astype(np.int64) > kth[1])))
