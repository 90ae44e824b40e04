"""frr_recheck_static: the entry point that allocates nothing.

It exists for callers that cannot let the library allocate device memory (a
latency-critical loop that must not stall the GPU in cudaMalloc / cudaFree, or an
application whose device memory belongs to another allocator). It runs the
exact-sum recheck on caller-owned device buffers with its scratch in a fixed array
inside the library, so its results must equal those of frr_recheck, call after call.
This file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_2501_07642_b300 import frr
from paper_2501_07642_b300.workloads import ar1_covariates

pytestmark = pytest.mark.gpu

REL_M64 = 1e-11  # the recheck tolerance used by the parity tests


def test_static_scratch_recheck_matches_frr_recheck_on_two_calls_in_a_row():
    import torch

    from paper_2501_07642_b300 import build
    build.build_library()
    L = frr.lib()
    n, d, seed = 300, 200, 41
    X = ar1_covariates(n, d, 77, 0.4)
    rng = np.random.default_rng(5)
    with frr.Context(X, n // 2, precision="f32", whiten="ridge") as ctx:
        # first call larger than the second: stale partial sums would show up in call two
        for count in (3000, 257):
            draws = rng.integers(0, 1 << 45, count).astype(np.uint64)
            want = frr.frr_recheck(ctx, seed, draws)
            d_draws = torch.from_numpy(draws.view(np.int64)).cuda()
            d_out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
            st = L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), count, d_out.data_ptr())
            assert st == frr.FRR_OK, frr.strerror(st)
            got = d_out.cpu().numpy()
            assert np.allclose(got, want, rtol=REL_M64, atol=0)

        # exactly as many partial sums as the fixed scratch holds: the last entries of the
        # array are written and read, and the result still equals frr_recheck
        ncb = -(-d // 128)
        full = 131072 // ncb
        draws = rng.integers(0, 1 << 45, full).astype(np.uint64)
        want = frr.frr_recheck(ctx, seed, draws)
        d_draws = torch.from_numpy(draws.view(np.int64)).cuda()
        d_out = torch.full((full,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), full, d_out.data_ptr())
        assert st == frr.FRR_OK, frr.strerror(st)
        assert np.allclose(d_out.cpu().numpy(), want, rtol=REL_M64, atol=0)

        # count == 0: nothing to do, the buffers stay untouched
        d_out = torch.full((2,), -7.0, dtype=torch.float64, device="cuda")
        assert L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), 0, d_out.data_ptr()) == frr.FRR_OK
        assert bool((d_out == -7.0).all())

        # beyond the fixed scratch: a clear error, nothing runs
        too_many = full + 1
        d_out = torch.zeros(1, dtype=torch.float64, device="cuda")
        d_draws = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), too_many, d_out.data_ptr()) == -6
        # host buffers, device buffers that are not 8-byte aligned (checked on the host, before
        # anything is launched) and exact-enumeration pools are refused
        h = np.zeros(4, dtype=np.uint64)
        ho = np.zeros(4)
        assert L.frr_recheck_static(ctx.handle, seed, h.ctypes.data, 4, ho.ctypes.data) == -1
        assert L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), 1, ho.ctypes.data) == -1
        d_big = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr(), 1, d_big.data_ptr() + 4) == -1
        assert L.frr_recheck_static(ctx.handle, seed, d_draws.data_ptr() + 4, 1, d_big.data_ptr()) == -1
        assert L.frr_recheck_static(ctx.handle, frr.FRR_EXACT_SEED, d_draws.data_ptr(), 1,
                                    d_out.data_ptr()) == -9
