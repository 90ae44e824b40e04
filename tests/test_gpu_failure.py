"""Failure path on the GPU without a fault: a bounded device wait that is never satisfied.

The balance kernel's covariate-tile producer is told to issue nothing (frr_test_wait_expiry),
so the MMA issuer's first wait for a tile can only expire. With the wait limit shortened to
about 2 ms the kernel must record the expired wait, release its tensor memory and return;
the call reports FRR_E_TIMEOUT within milliseconds, the context stays usable, and a fresh
context on the same GPU still reproduces the oracle's accepted pool. Nothing traps, faults or
waits without a limit.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import ar1_covariates

pytestmark = pytest.mark.gpu

FRR_E_TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_07642_b300 import build
    build.build_library()
    O.build()


def _oracle_pool(X, n1, seed, B, q):
    Zc, *_ = O.prep(X, "chol")
    return O.select(Zc, n1, seed, 0, B, q=q)


@pytest.mark.parametrize("n,d", [(300, 200), (1000, 600)])
def test_expired_wait_returns_timeout_and_the_gpu_stays_usable(n, d):
    X = ar1_covariates(n, d, 90 + n, 0.3)
    n1, seed, B, q = n // 2, 17, 30_000, 0.01
    want_keys, want_m = _oracle_pool(X, n1, seed, B, q)
    with frr.Context(X, n1, precision="split_bf16", whiten="chol") as ctx:
        t0 = time.perf_counter()
        st = frr.frr_test_wait_expiry(ctx, 1 << 22)
        dt = time.perf_counter() - t0
        assert st == FRR_E_TIMEOUT, frr.strerror(st)
        assert dt < 0.5, dt
        # the expired wait was cleared and the context still works: same pool as the oracle
        keys, m64 = frr.frr_select(ctx, seed, 0, B, q=q)
        assert np.array_equal(keys, want_keys)
        assert np.allclose(m64, want_m, rtol=1e-11, atol=0)
        # a second expiry in a row behaves the same
        assert frr.frr_test_wait_expiry(ctx, 1 << 20) == FRR_E_TIMEOUT
    # a fresh context on the same GPU after the destroyed one
    with frr.Context(X, n1, precision="split_bf16", whiten="chol") as ctx:
        keys, m64 = frr.frr_select(ctx, seed, 0, B, q=q)
    assert np.array_equal(keys, want_keys)
    assert np.allclose(m64, want_m, rtol=1e-11, atol=0)


def test_expired_wait_is_refused_for_the_fp32_path():
    X = ar1_covariates(64, 8, 3, 0.0)
    with frr.Context(X, 32, precision="f32", whiten="chol") as ctx:
        assert frr.frr_test_wait_expiry(ctx, 1 << 22) == -9
