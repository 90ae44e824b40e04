// frr_diag.cu -- planning diagnostics (Sec. 2.2 "Choosing stringency"; App. A-D).
//
// Scalar host code: a handful of chi-square and normal distribution evaluations per
// call, nothing data-parallel. Notation as in the paper, k = 1/n_T + 1/n_C:
//   realised RMSE (typical orientation, App. A)  sqrt(sigma^2 k + sigma_prog^2 M / d)
//   Cauchy-Schwarz bound (App. A)                sqrt(sigma^2 k + sigma_prog^2 M)
//   sigma_prog^2 = R^2 / (1 - R^2) sigma^2       (Sec. 2.2 definition of R^2)
//   c_q = chi2_d quantile at q, a_q = k c_q      (Sec. 2.2)
//   v_a = P(chi2_{d+2} <= c_q) / q               (App. C)
//   RMSE(q) = sqrt(k (sigma^2 + v_a sigma_prog^2)), E[M | accept] = k d v_a   (App. C)
//   q* = largest q with RMSE(q) <= |tau| / (z_{1-alpha/2} + z_power)        (App. D)
//
// The chi-square CDF is the regularised lower incomplete gamma P(d/2, c/2), kept in
// logarithms so that the far lower tail (q far below 1e-300 is possible at large d)
// stays representable: the power series for x < a + 1, otherwise 1 - Q with Q from
// Legendre's continued fraction, evaluated by the modified Lentz algorithm (Lentz,
// Appl. Opt. 15, 1976; Thompson & Barnett, J. Comput. Phys. 64, 1986). The normal CDF
// is erfc from the C library; quantiles are found by safeguarded Newton iterations.
#include <math.h>
#include <float.h>
#include <stdint.h>

#include "../../include/frr.h"

namespace {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kSqrt2 = 1.41421356237309504880;

// log P(a, x), a > 0
double log_gamma_p(double a, double x)
{
    if (!(x > 0.0)) return -INFINITY;
    if (isinf(x)) return 0.0;
    const double lpre = a * log(x) - x;
    if (x < a + 1.0) {
        // P = x^a e^-x / Gamma(a + 1) * sum_k x^k / ((a + 1) ... (a + k))
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < 100000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (term < sum * 1e-17) break;
        }
        return lpre - lgamma(a + 1.0) + log(sum);
    }
    // Q = x^a e^-x / Gamma(a) * 1 / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / ...))
    const double tiny = 1e-300;
    double b = x + 1.0 - a;
    double c = 1.0 / tiny;
    double dd = 1.0 / b;
    double h = dd;
    for (int i = 1; i < 100000; ++i) {
        const double an = -i * (i - a);
        b += 2.0;
        dd = an * dd + b;
        if (fabs(dd) < tiny) dd = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        dd = 1.0 / dd;
        const double del = dd * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    const double Q = exp(lpre - lgamma(a)) * h;
    return log1p(-Q);
}

// log P(chi2_d <= c)
double chi2_logcdf(double c, double d) { return log_gamma_p(0.5 * d, 0.5 * c); }

// log of the chi2_d density at c > 0
double chi2_logpdf(double c, double d)
{
    return (0.5 * d - 1.0) * log(c) - 0.5 * c - 0.5 * d * kLn2 - lgamma(0.5 * d);
}

// v_a at the chi-square cut c (App. C), as a ratio of log-CDFs
double v_of_c(double c, double d)
{
    if (isinf(c)) return 1.0;
    return exp(chi2_logcdf(c, d + 2.0) - chi2_logcdf(c, d));
}

// chi2_d quantile at log-probability lq < 0: Newton on log P with a bisection safeguard
double chi2_quantile_log(double lq, double d)
{
    double lo = 0.0, hi = d > 1.0 ? d : 1.0;
    for (int i = 0; i < 2000 && chi2_logcdf(hi, d) < lq; ++i) hi *= 2.0;
    double c = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        const double g = chi2_logcdf(c, d) - lq;
        if (g == 0.0) return c;
        if (g > 0.0) hi = c; else lo = c;
        const double step = g / exp(chi2_logpdf(c, d) - chi2_logcdf(c, d));
        double next = c - step;
        if (!(next > lo && next < hi)) next = lo > 0.0 ? sqrt(lo * hi) : 0.5 * hi;
        if (fabs(next - c) <= 1e-16 * c || hi - lo <= 1e-16 * hi) return next;
        c = next;
    }
    return c;
}

double norm_cdf(double z) { return 0.5 * erfc(-z / kSqrt2); }

// z with Phi(z) = p, 0 < p < 1
double norm_quantile(double p)
{
    double lo = -40.0, hi = 40.0, z = 0.0;
    const double inv_sqrt_2pi = 0.39894228040143267794;
    for (int it = 0; it < 200; ++it) {
        const double g = norm_cdf(z) - p;
        if (g == 0.0) return z;
        if (g > 0.0) hi = z; else lo = z;
        const double pdf = inv_sqrt_2pi * exp(-0.5 * z * z);
        double next = pdf > 0.0 ? z - g / pdf : 0.5 * (lo + hi);
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (fabs(next - z) <= 1e-15 * (1.0 + fabs(z))) return next;
        z = next;
    }
    return z;
}

}  // namespace

extern "C" frr_status frr_diagnose(const frr_diag_in* in, frr_diag_out* out)
{
    if (in == nullptr || out == nullptr) return FRR_E_ARG;
    const frr_diag_in p = *in;
    const bool has_q = !isnan(p.q), has_M = !isnan(p.M_obs), has_tau = !isnan(p.tau);
    if (p.n_T < 1 || p.n_C < 1 || p.d < 1) return FRR_E_ARG;
    if (!(p.R2 >= 0.0 && p.R2 < 1.0) || !(p.sigma > 0.0) || !isfinite(p.sigma)) return FRR_E_ARG;
    if (has_q && !(p.q > 0.0 && p.q <= 1.0)) return FRR_E_ARG;
    if (has_M && !(p.M_obs >= 0.0 && isfinite(p.M_obs))) return FRR_E_ARG;
    if (has_tau && (!isfinite(p.tau) || !(p.alpha > 0.0 && p.alpha < 1.0) || !(p.power > 0.0 && p.power < 1.0)))
        return FRR_E_ARG;

    frr_diag_out o;
    o.k = o.sigma2_prog = o.rmse_complete = NAN;
    o.rmse_realised = o.rmse_cs_bound = NAN;
    o.c_q = o.a_q = o.v_a = o.rmse_accept = o.rmse_reduction = o.expected_M = o.power_at_q = NAN;
    o.snr_needed = o.q_star = o.log10_q_star = o.c_star = o.v_star = o.draws_per_accept = NAN;
    o.q_star_status = -1;

    const double d = (double)p.d, s2 = p.sigma * p.sigma;
    o.k = 1.0 / (double)p.n_T + 1.0 / (double)p.n_C;
    o.sigma2_prog = p.R2 / (1.0 - p.R2) * s2;
    o.rmse_complete = sqrt(o.k * (s2 + o.sigma2_prog));
    if (has_M) {
        o.rmse_realised = sqrt(s2 * o.k + o.sigma2_prog * p.M_obs / d);
        o.rmse_cs_bound = sqrt(s2 * o.k + o.sigma2_prog * p.M_obs);
    }
    double z_half = NAN;
    if (has_tau) {
        z_half = norm_quantile(1.0 - 0.5 * p.alpha);
        o.snr_needed = z_half + norm_quantile(p.power);
    }
    if (has_q) {
        o.c_q = p.q >= 1.0 ? INFINITY : chi2_quantile_log(log(p.q), d);
        o.a_q = o.k * o.c_q;
        o.v_a = v_of_c(o.c_q, d);
        o.rmse_accept = sqrt(o.k * (s2 + o.v_a * o.sigma2_prog));
        o.rmse_reduction = 1.0 - o.rmse_accept / o.rmse_complete;
        o.expected_M = o.k * d * o.v_a;
        if (has_tau) {
            const double s = fabs(p.tau) / o.rmse_accept;
            o.power_at_q = norm_cdf(s - z_half) + norm_cdf(-s - z_half);
        }
    }
    if (has_tau) {
        const double target2 = (p.tau / o.snr_needed) * (p.tau / o.snr_needed);
        if (target2 <= s2 * o.k) {
            o.q_star_status = 2;                       // the irreducible term alone misses the target
        } else {
            const double v_need = o.sigma2_prog > 0.0 ? (target2 / o.k - s2) / o.sigma2_prog : INFINITY;
            if (v_need >= 1.0) {
                o.q_star_status = 1;                   // complete randomization already meets it
                o.q_star = 1.0;
                o.log10_q_star = 0.0;
                o.c_star = INFINITY;
                o.v_star = 1.0;
                o.draws_per_accept = 1.0;
            } else {
                // line search over the chi-square cut c, where v_a increases (App. D);
                // v_a(c) <= c / d brackets it from below
                double lo = 0.5 * v_need * d, hi = 2.0 * d;
                for (int i = 0; i < 2000 && v_of_c(hi, d) < v_need; ++i) hi *= 2.0;
                for (int it = 0; it < 400 && hi - lo > 1e-16 * hi; ++it) {
                    const double mid = sqrt(lo * hi);
                    if (mid <= lo || mid >= hi) break;
                    if (v_of_c(mid, d) < v_need) lo = mid; else hi = mid;
                }
                const double c = sqrt(lo * hi);
                const double lq = chi2_logcdf(c, d);
                o.q_star_status = 0;
                o.c_star = c;
                o.v_star = v_of_c(c, d);
                o.log10_q_star = lq / log(10.0);
                o.q_star = exp(lq);                    // 0 when below the double range
                o.draws_per_accept = exp(-lq);         // inf then
            }
        }
    }
    *out = o;
    return FRR_OK;
}
