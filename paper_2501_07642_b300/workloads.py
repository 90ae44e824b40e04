"""Seeded synthetic inputs shaped like the paper's rerandomization workloads.

This module only draws random numbers. It holds none of the method's
arithmetic (no centring, whitening, balance, selection or test statistic), so
both the CUDA path and the FP64 oracle may take their inputs from it.

Shapes follow the benchmarks of Sec. 4 ("Impact": n in {100, 1000},
d in {100, 1000}, q in {0.01, 0.005, 0.00025}, 1e5 / 2e5 draws), the Gaussian
covariates of the usage example in the "Sample code snippets" appendix, and the
linear outcome model Y_i(t) = beta^T X_i + tau t + eps_i of Sec. 2.2 /
Appendix A. The paper names no public dataset; its CLIP satellite-embedding
example (Sec. 3) is not available, and these synthetic matrices stand in for it.

Every generator is ``numpy.random.default_rng(seed)`` in FP64, row-major
(units are rows), and the draw order inside a recipe is fixed as written.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "ar1_covariates",
    "mixed_standardised_covariates",
    "outcome",
    "workload",
    "batched_workloads",
    "WORKLOADS",
]


def ar1_covariates(n: int, d: int, seed, rho: float) -> np.ndarray:
    """X = G chol(Sigma)^T with Sigma_jk = rho^|j-k| and G iid N(0,1) (n x d)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, d))
    if rho == 0.0:
        return np.ascontiguousarray(g)
    idx = np.arange(d)
    sigma = rho ** np.abs(idx[:, None] - idx[None, :])
    chol = np.linalg.cholesky(sigma)
    return np.ascontiguousarray(g @ chol.T)


def mixed_standardised_covariates(n: int, d: int, seed) -> np.ndarray:
    """Half N(0,1), a quarter Bernoulli(0.3), a quarter lognormal(0,1) columns,
    each then standardised to mean 0, sd 1 (ddof=1).

    Draw order: the normal block, then the uniforms behind the Bernoulli block,
    then the normals behind the lognormal block.
    """
    rng = np.random.default_rng(seed)
    d_norm = d // 2
    d_bern = d // 4
    d_logn = d - d_norm - d_bern
    a = rng.standard_normal((n, d_norm))
    b = (rng.random((n, d_bern)) < 0.3).astype(np.float64)
    c = np.exp(rng.standard_normal((n, d_logn)))
    x = np.hstack([a, b, c])
    mu = x.mean(axis=0)
    sd = x.std(axis=0, ddof=1)
    sd[sd == 0.0] = 1.0  # a constant Bernoulli column (vanishingly rare) stays constant
    return np.ascontiguousarray((x - mu) / sd)


def outcome(x: np.ndarray, w_obs: np.ndarray, tau: float, seed, noise_sd: float = 1.0) -> np.ndarray:
    """Y = X beta + tau * w_obs + noise_sd * eps with beta ~ N(0, I_d), eps ~ N(0, I_n).

    Draw order: beta, then eps.
    """
    rng = np.random.default_rng(seed)
    n, d = x.shape
    beta = rng.standard_normal(d)
    eps = rng.standard_normal(n)
    return np.ascontiguousarray(x @ beta + tau * np.asarray(w_obs, dtype=np.float64) + noise_sd * eps)


@dataclass
class Workload:
    """One experiment: covariates plus the draw / acceptance parameters."""

    name: str
    n: int
    n1: int
    d: int
    x_seed: object
    kind: str  # "gauss", "ar1", "mixed"
    rho: float = 0.0
    philox_seed: int | None = None  # None = exact enumeration
    draws: int = 0
    q: float | None = None
    whiten: str = "chol"  # "chol" | "ridge" | "diag"
    ridge: float = 0.0
    y_seed: object = None
    tau_true: float = 0.0
    noise_sd: float = 1.0
    tau_grid: np.ndarray | None = field(default=None, repr=False)
    chunk: int | None = None

    def covariates(self) -> np.ndarray:
        if self.kind == "mixed":
            return mixed_standardised_covariates(self.n, self.d, self.x_seed)
        return ar1_covariates(self.n, self.d, self.x_seed, self.rho)


def _whiten_rule(n: int, d: int) -> tuple[str, float]:
    # Full Mahalanobis is degenerate once d >= n-1 (every assignment has M = n-1);
    # the stated reading is a ridge of 0.1 * tr(S)/d there.
    return ("chol", 0.0) if d <= n - 2 else ("ridge", 0.1)


def workload(name: str) -> Workload:
    """The five named workloads (exact, plain FP32, precision, batched, streaming)."""
    if name == "exact_n20_d5":
        return Workload(name, 20, 10, 5, 0, "gauss", philox_seed=None,
                        draws=math.comb(20, 10), q=0.05, whiten="chol", y_seed=10,
                        tau_true=1.0, noise_sd=1.0,
                        tau_grid=np.round(np.linspace(-1.0, 3.0, 201), 12))
    if name == "mc_n100_d100":
        return Workload(name, 100, 50, 100, 102, "ar1", rho=0.5, philox_seed=1,
                        draws=200_000, q=0.01, whiten="ridge", ridge=0.1, y_seed=202,
                        tau_true=0.2, noise_sd=1.0,
                        tau_grid=np.round(-1.0 + 0.01 * np.arange(201), 12))
    if name == "precision_n1000_d1000":
        return Workload(name, 1000, 500, 1000, 103, "mixed", philox_seed=3,
                        draws=200_000, q=1e-3, whiten="ridge", ridge=0.1)
    if name == "stream_n1000_d1000":
        return Workload(name, 1000, 500, 1000, 105, "ar1", rho=0.5, philox_seed=5,
                        draws=100_000_000, q=1.2e-5, whiten="ridge", ridge=0.1,
                        chunk=1_000_000)
    raise KeyError(name)


def batched_workloads(count: int = 256) -> list[Workload]:
    """Experiment e: n log-uniform on [50, 2000], n1 = n // 2, d uniform on {10..500},
    X ~ N(0, AR(1) rho=0.3), 1e5 draws, q = 0.01. Sizes drawn from default_rng([104, e])
    before the covariates (which use default_rng([1104, e]))."""
    out = []
    for e in range(count):
        rng = np.random.default_rng([104, e])
        n = int(math.floor(math.exp(rng.uniform(math.log(50.0), math.log(2000.0)))))
        d = int(rng.integers(10, 501))
        wh, lam = _whiten_rule(n, d)
        out.append(Workload(f"batched_{e}", n, n // 2, d, [1104, e], "ar1", rho=0.3,
                            philox_seed=(4 << 32) + e, draws=100_000, q=0.01,
                            whiten=wh, ridge=lam, y_seed=[204, e], tau_true=0.2,
                            tau_grid=np.round(-1.0 + 0.01 * np.arange(201), 12)))
    return out


WORKLOADS = ("exact_n20_d5", "mc_n100_d100", "precision_n1000_d1000", "stream_n1000_d1000")
