"""Tight-threshold streaming workload: n = d = 1000, AR(1) rho = 0.5 covariates,
1e8 Philox draws streamed in 1e6-draw chunks, q = 1.2e-5 (K = 1200), split-BF16 bulk
path with the exact recheck. The oracle re-scores every accepted key and a seeded
sample of 1e5 draws; every sampled rejected draw must come after the last accepted one
in (M, draw index). A checkpoint saved after chunk 37 and restored into a fresh context
must finish with exactly the same accepted keys and M64."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import ar1_covariates, workload

pytestmark = pytest.mark.gpu

STOP = 37  # chunks streamed before the checkpoint


@pytest.fixture(scope="module")
def stream_run():
    from paper_2501_07642_b300 import build
    build.build_library()
    w = workload("stream_n1000_d1000")
    X = w.covariates()
    with frr.Context(X, w.n1, precision="split_bf16", whiten=w.whiten, ridge=w.ridge) as ctx:
        frr.frr_stream_begin(ctx, w.philox_seed, w.draws, q=w.q)
        blob = None
        for c in range(w.draws // w.chunk):
            frr.frr_stream_chunk(ctx, c * w.chunk, w.chunk)
            if c + 1 == STOP:
                blob = frr.frr_stream_save(ctx)
        keys, m64 = frr.frr_stream_end(ctx, 4096)
        st = frr.frr_last_stats(ctx)
    return w, X, keys, m64, st, blob


def test_stream_1e8_draws_in_1e6_chunks(stream_run):
    w, X, keys, m64, st, _ = stream_run
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


def test_stream_resumes_from_a_checkpoint_in_a_fresh_context(stream_run):
    w, X, keys, m64, _, blob = stream_run
    info = frr.frr_stream_blob_info(blob)
    assert info["seen"] == STOP * w.chunk and info["total"] == w.draws and info["K"] == 1200
    assert len(blob) == 256 + 12 * info["retained"]
    with frr.Context(X, w.n1, precision="split_bf16", whiten=w.whiten, ridge=w.ridge) as ctx:
        frr.frr_stream_load(ctx, blob)
        for c in range(STOP, w.draws // w.chunk):
            frr.frr_stream_chunk(ctx, c * w.chunk, w.chunk)
        k2, m2 = frr.frr_stream_end(ctx, 4096)
        st = frr.frr_last_stats(ctx)
        with pytest.raises(frr.FrrError) as e:  # no stream is running after frr_stream_end
            frr.frr_stream_save(ctx)
        assert e.value.name == "FRR_E_STATE"
    assert np.array_equal(k2, keys) and np.array_equal(m2, m64)
    assert st["draws"] == w.draws and st["band_violations"] == 0
    # a context of the same shape prepared from other covariates, and one of the other bulk
    # path, refuse the blob (their error bands differ)
    X2 = ar1_covariates(w.n, w.d, 7, 0.5)
    with frr.Context(X2, w.n1, precision="split_bf16", whiten=w.whiten, ridge=w.ridge) as ctx:
        with pytest.raises(frr.FrrError) as e:
            frr.frr_stream_load(ctx, blob)
        assert e.value.name == "FRR_E_ARG"
    with frr.Context(X, w.n1, precision="f32", whiten=w.whiten, ridge=w.ridge) as ctx:
        with pytest.raises(frr.FrrError) as e:
            frr.frr_stream_load(ctx, blob)
        assert e.value.name == "FRR_E_ARG"


def test_checkpoint_round_trip_in_the_same_context_small():
    """Save after every chunk of a small threshold-mode stream and reload each blob into
    the same context before the next chunk: the result equals one frr_select."""
    X = ar1_covariates(200, 50, 21, 0.3)
    with frr.Context(X, 100, precision="split_bf16", whiten="chol") as ctx:
        k1, m1 = frr.frr_select(ctx, 9, 0, 60_000, q=0.004)
        a = float(m1.max())
        k1, m1 = frr.frr_select(ctx, 9, 0, 60_000, threshold=a)
        frr.frr_stream_begin(ctx, 9, 60_000, threshold=a)
        for c in range(6):
            frr.frr_stream_chunk(ctx, c * 10_000, 10_000)
            blob = frr.frr_stream_save(ctx)
            frr.frr_stream_load(ctx, blob)
        k2, m2 = frr.frr_stream_end(ctx, 4096)
    assert np.array_equal(k1, k2) and np.array_equal(m1, m2)
