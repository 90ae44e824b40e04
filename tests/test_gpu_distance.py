"""Pairwise distances on the tensor cores (Sec. 4, fast_distance) against the FP64 oracle.

Bound (from the arithmetic: two BF16 parts per value, FP32 accumulation over 3 dp terms,
FP32 norms and epilogue): |D^2 - exact| <= (3 * 2^-18 + (3 dp + 4) * 2^-24 + 2^-22)
(|x|^2 + |y|^2), dp = d rounded up to 64; the 2^-22 term covers the rounding of the
square root when D itself is returned.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_07642_b300 import frr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_07642_b300 import build
    build.build_library()
    O.build()


def _bound(d):
    dp = 64 * math.ceil(d / 64)
    return 3 * 2.0 ** -18 + (3 * dp + 4) * 2.0 ** -24 + 2.0 ** -22


def _check(X, Y, D, squared):
    want = O.distance(X, Y, squared=True)
    got2 = D.astype(np.float64) if squared else D.astype(np.float64) ** 2
    Yr = X if Y is None else Y
    scale = (X.astype(np.float64) ** 2).sum(1)[:, None] + (Yr.astype(np.float64) ** 2).sum(1)[None, :]
    err = np.abs(got2 - want) / np.maximum(scale, 1e-300)
    assert err.max() <= _bound(X.shape[1]), err.max()
    return err.max()


# m % 4 == 0 takes the TMA-store epilogue, other m the direct stores
@pytest.mark.parametrize("n,m,d", [(300, 516, 77), (300, 517, 77), (128, 256, 64), (1, 1, 1), (1, 4, 3),
                                   (129, 260, 130), (129, 257, 130), (513, 3, 1000), (257, 1028, 200)])
@pytest.mark.parametrize("squared", [False, True])
def test_ragged_shapes_against_oracle(n, m, d, squared):
    rng = np.random.default_rng(n * 7 + m + d)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = (rng.standard_normal((m, d)) * 2 + 0.5).astype(np.float32)
    D = frr.frr_fast_distance(X, Y, squared=squared)
    assert D.shape == (n, m) and np.isfinite(D).all() and (D >= 0).all()
    _check(X, Y, D, squared)


def test_self_distance_symmetric_and_near_zero_diagonal():
    X = np.random.default_rng(5).standard_normal((400, 96)).astype(np.float32)
    D2 = frr.frr_fast_distance(X, None, squared=True)
    _check(X, None, D2, True)
    nrm = (X.astype(np.float64) ** 2).sum(1)
    assert np.all(np.diag(D2) <= _bound(96) * 2 * nrm)
    # the two operand layouts differ, so symmetry holds within the bound, not bit for bit
    assert np.all(np.abs(D2 - D2.T) <= 2 * _bound(96) * (nrm[:, None] + nrm[None, :]))


def test_device_buffers_and_unaligned_output():
    import torch
    rng = np.random.default_rng(9)
    X = rng.standard_normal((200, 50)).astype(np.float32)
    Y = rng.standard_normal((301, 50)).astype(np.float32)
    host = frr.frr_fast_distance(X, Y)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    Dd = torch.empty(200 * 301 + 1, dtype=torch.float32, device="cuda")
    view = Dd[1:]                       # 4-byte offset: the kernel falls back to scalar stores
    frr.frr_fast_distance(Xd, Yd, D_out=view)
    assert np.array_equal(view.cpu().numpy().reshape(200, 301), host)


def test_embedding_workload_sampled():
    # n = m = 16384 points of d = 768 (the CLIP embedding width of Sec. 3); 1 GiB of output
    import torch
    n, d = 16384, 768
    rng = np.random.default_rng(768)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = (rng.standard_normal((n, d)) * 0.5 + 0.1).astype(np.float32)
    Dd = torch.empty((n, n), dtype=torch.float32, device="cuda")
    frr.frr_fast_distance(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), D_out=Dd)
    ij = np.stack([rng.integers(0, n, 20000), rng.integers(0, n, 20000)], axis=1)
    got = Dd[torch.from_numpy(ij[:, 0]).cuda(), torch.from_numpy(ij[:, 1]).cuda()].cpu().numpy().astype(np.float64)
    want2 = O.distance_pairs(X, Y, ij, squared=True)
    scale = (X[ij[:, 0]].astype(np.float64) ** 2).sum(1) + (Y[ij[:, 1]].astype(np.float64) ** 2).sum(1)
    assert (np.abs(got ** 2 - want2) / scale).max() <= _bound(d)


def test_large_magnitudes_long_rows_and_mixed_buffers():
    import torch
    rng = np.random.default_rng(2048)
    X = (rng.standard_normal((150, 2048)) * 3e3 + 1e3).astype(np.float32)
    Y = (rng.standard_normal((70, 2048)) * 3e3).astype(np.float32)
    Dd = torch.empty((150, 70), dtype=torch.float32, device="cuda")
    frr.frr_fast_distance(X, Y, D_out=Dd)          # host inputs, device output
    _check(X, Y, Dd.cpu().numpy(), False)
    D2 = frr.frr_fast_distance(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), squared=True)  # device in, host out
    _check(X, Y, D2, True)


def test_duplicate_rows_give_near_zero_distances():
    rng = np.random.default_rng(4)
    base = rng.standard_normal((40, 300)).astype(np.float32)
    X = np.concatenate([base, base[::-1]])
    D2 = frr.frr_fast_distance(X, None, squared=True)
    nrm = (X.astype(np.float64) ** 2).sum(1)
    for i in range(40):
        j = 79 - i                                   # the duplicate of row i
        assert D2[i, j] >= 0.0 and D2[i, j] <= _bound(300) * 2 * nrm[i]
