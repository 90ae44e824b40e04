"""Oracle for the planning diagnostics (Sec. 2.2 "Choosing stringency"; App. A-D).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package. It
shares no code with the CUDA library's host implementation (frr_diagnose) and
does not import it. Library primitives serve as steps: scipy's chi-square quantile
and normal distribution functions, a bracketing root finder, and mpmath's regularised
incomplete gamma function at 40 significant digits for the chi-square CDF (its far
lower tail, which the q* search reaches at large d, is below the double range).

Quantities, in the paper's notation (k = 1/n_T + 1/n_C):
  App. A   realised RMSE, typical orientation   sqrt(sigma^2 k + sigma_prog^2 M / d)
           Cauchy-Schwarz upper bound           sqrt(sigma^2 k + sigma_prog^2 M)
           sigma_prog^2 = R^2 / (1 - R^2) sigma^2
  Sec. 2.2 c_q = chi2_d quantile at q, a_q = k c_q
  App. C   v_a(d) = P(chi2_{d+2} <= c_q) / P(chi2_d <= c_q)
           ex-ante MSE given acceptance = k (sigma^2 + v_a sigma_prog^2)
           E[M | accept] = k d v_a
  App. B   complete randomization: k (sigma^2 + sigma_prog^2)
  App. D   snr_needed = z_{1-alpha/2} + z_{power}; q* = largest q with
           RMSE(q) <= |tau| / snr_needed (a line search; v_a increases with q)
  App. D footnote: two-sided power P(|Z + tau/RMSE| > z_{1-alpha/2}).

Pins (tests/test_diag.py): the paper's printed v_a and RMSE reductions, the
closed forms of the chi-square CDF at d = 2 and 4, numerical integration of the
truncated first moment, a Monte Carlo check of the 1/d orientation factor, and
textbook normal quantiles.
"""
from __future__ import annotations

import math

import mpmath
from scipy import optimize, stats


def k_factor(n_T: int, n_C: int) -> float:
    return 1.0 / n_T + 1.0 / n_C


def sigma2_prog(R2: float, sigma: float) -> float:
    """Prognostic variance from the share R^2 (Sec. 2.2 definition of R^2)."""
    return R2 / (1.0 - R2) * sigma * sigma


def rmse_realised(n_T, n_C, d, R2, sigma, M) -> float:
    """Typical-orientation RMSE given the observed M (Sec. 2.2; App. A item 2)."""
    return math.sqrt(sigma * sigma * k_factor(n_T, n_C) + sigma2_prog(R2, sigma) * M / d)


def rmse_cs_bound(n_T, n_C, d, R2, sigma, M) -> float:
    """Cauchy-Schwarz upper bound on the realised RMSE (App. A item 1)."""
    return math.sqrt(sigma * sigma * k_factor(n_T, n_C) + sigma2_prog(R2, sigma) * M)


def c_of_q(d: int, q: float) -> float:
    """chi2_d quantile c_q (Sec. 2.2)."""
    return float(stats.chi2.ppf(q, d))


def chi2_cdf_mp(c: float, d: int):
    """P(chi2_d <= c) = P(d/2, c/2), regularised lower incomplete gamma, as an mpmath number."""
    with mpmath.workdps(40):
        return mpmath.gammainc(mpmath.mpf(d) / 2, 0, mpmath.mpf(c) / 2, regularized=True)


def chi2_logcdf(c: float, d: int) -> float:
    if math.isinf(c):
        return 0.0
    with mpmath.workdps(40):
        return float(mpmath.log(chi2_cdf_mp(c, d)))


def v_a_of_c(d: int, c: float) -> float:
    """Shrinkage factor v_a(d) at chi-square cut c (App. C): P(chi2_{d+2} <= c) / P(chi2_d <= c)."""
    if math.isinf(c):
        return 1.0
    with mpmath.workdps(40):
        return float(chi2_cdf_mp(c, d + 2) / chi2_cdf_mp(c, d))


def v_a(d: int, q: float) -> float:
    return v_a_of_c(d, c_of_q(d, q))


def rmse_complete(n_T, n_C, R2, sigma) -> float:
    """Ex-ante RMSE under complete randomization (App. B)."""
    return math.sqrt(k_factor(n_T, n_C) * (sigma * sigma + sigma2_prog(R2, sigma)))


def rmse_accept(n_T, n_C, d, R2, sigma, q) -> float:
    """Ex-ante RMSE conditional on acceptance at probability q (App. C)."""
    return math.sqrt(k_factor(n_T, n_C) * (sigma * sigma + v_a(d, q) * sigma2_prog(R2, sigma)))


def expected_M(n_T, n_C, d, q) -> float:
    """E[M | accept] = k d v_a (App. C, trace identity)."""
    return k_factor(n_T, n_C) * d * v_a(d, q)


def snr_needed(alpha: float, power: float) -> float:
    """z_{1-alpha/2} + z_{power} (App. D)."""
    return float(stats.norm.ppf(1.0 - alpha / 2.0) + stats.norm.ppf(power))


def power_two_sided(tau: float, rmse: float, alpha: float) -> float:
    """P(|Z + tau/RMSE| > z_{1-alpha/2}), Z ~ N(0, 1) (App. D footnote)."""
    z = stats.norm.ppf(1.0 - alpha / 2.0)
    s = abs(tau) / rmse
    return float(stats.norm.sf(z - s) + stats.norm.cdf(-z - s))


def q_star(n_T, n_C, d, R2, sigma, tau, alpha, power):
    """Largest acceptance probability meeting the power target (App. D).

    Returns (status, log_q, c): status 0 = found by the line search, 1 = q = 1 already
    meets the target, 2 = unreachable (the irreducible term alone exceeds the target).
    The search runs over the chi-square cut c, where v_a is increasing; q = P(chi2_d <= c)
    is reported through its logarithm because it can fall below the double range.
    """
    k = k_factor(n_T, n_C)
    s2p = sigma2_prog(R2, sigma)
    target2 = (abs(tau) / snr_needed(alpha, power)) ** 2
    if target2 <= sigma * sigma * k:
        return 2, float("nan"), float("nan")
    if s2p == 0.0:
        return 1, 0.0, float("inf")
    v_need = (target2 / k - sigma * sigma) / s2p
    if v_need >= 1.0:
        return 1, 0.0, float("inf")
    f = lambda lc: v_a_of_c(d, math.exp(lc)) - v_need
    lo = math.log(0.5 * v_need * d)      # v_a(c) <= c / d
    hi = math.log(max(2.0 * d, 1.0))
    while f(hi) < 0.0:
        hi += 1.0
    lc = optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    c = math.exp(lc)
    return 0, chi2_logcdf(c, d), c


def diagnose(n_T, n_C, d, R2, sigma, q=float("nan"), M_obs=float("nan"), tau=float("nan"),
             alpha=0.05, power=0.8) -> dict:
    """All diagnostics of one call, keyed like the library's output record."""
    out = {"k": k_factor(n_T, n_C), "sigma2_prog": sigma2_prog(R2, sigma)}
    if not math.isnan(M_obs):
        out["rmse_realised"] = rmse_realised(n_T, n_C, d, R2, sigma, M_obs)
        out["rmse_cs_bound"] = rmse_cs_bound(n_T, n_C, d, R2, sigma, M_obs)
    out["rmse_complete"] = rmse_complete(n_T, n_C, R2, sigma)
    if not math.isnan(q):
        c = c_of_q(d, q)
        va = v_a_of_c(d, c)
        out.update(c_q=c, a_q=out["k"] * c, v_a=va,
                   rmse_accept=math.sqrt(out["k"] * (sigma * sigma + va * out["sigma2_prog"])),
                   expected_M=out["k"] * d * va)
        out["rmse_reduction"] = 1.0 - out["rmse_accept"] / out["rmse_complete"]
        if not math.isnan(tau):
            out["power_at_q"] = power_two_sided(tau, out["rmse_accept"], alpha)
    if not math.isnan(tau):
        out["snr_needed"] = snr_needed(alpha, power)
        st, lq, c = q_star(n_T, n_C, d, R2, sigma, tau, alpha, power)
        out["q_star_status"] = st
        out["log_q_star"] = lq
        out["c_star"] = c
    return out
