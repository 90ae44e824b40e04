// frr_prep.cu -- FP64 preparation of an experiment on the GPU (runs once per frr_init).
//
// Sec. 2.2 works with covariates that are centred and whitened so that the
// Mahalanobis distance is Euclidean (App. A, remark on general Sigma_X):
//   xbar = column means, Xc = X - 1 xbar^T, S = Xc^T Xc / (n - 1),
//   S_lambda = S (+ ridge * tr(S)/d * I), S_lambda = L L^T, Zc = Xc L^{-T}.
// Every step uses explicitly rounded FP64 operations (no contraction into
// FMA) in ascending index order, one dependent chain per output, so the
// results do not depend on the launch shape.
//
// From Zc (natural unit order) the kernels below derive the arrays the
// balance path reads, all in K-order (see frr_gen.cuh):
//   Z32  : FP32 copy for the SIMT path,
//   Zhi, Zlo : BF16 hi/lo split (Zc ~ hi + lo) for the tensor-core path,
//   Q    : fixed-point Zc * 2^qexp_j (int64) for the exact-sum recheck,
//   band : per-column error-band terms of both bulk paths.
#include "frr_internal.cuh"
#include "frr_gen.cuh"

#include <vector>

namespace frr {
namespace {

__global__ void k_colmean(const double* __restrict__ X, int n, int d, double* __restrict__ xbar)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = __dadd_rn(s, X[(size_t)i * d + j]);
    xbar[j] = __ddiv_rn(s, (double)n);
}

__global__ void k_center(const double* __restrict__ X, const double* __restrict__ xbar, int n, int d,
                         double* __restrict__ Xc)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * d) return;
    Xc[idx] = __dsub_rn(X[idx], xbar[idx % d]);
}

// S_jk = sum_i Xc_ij Xc_ik / (n - 1) for k >= j, mirrored (the product is commutative,
// so both halves are the value a separate (k, j) computation would give).
__global__ void k_cov(const double* __restrict__ Xc, int n, int d, double* __restrict__ S)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= d || k >= d || k < j) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = __dadd_rn(s, __dmul_rn(Xc[(size_t)i * d + j], Xc[(size_t)i * d + k]));
    const double v = __ddiv_rn(s, (double)(n - 1));
    S[(size_t)j * d + k] = v;
    S[(size_t)k * d + j] = v;
}

// trace, max diagonal, and the diagonal of S_lambda (ridge added)
__global__ void k_diag(const double* __restrict__ S, int d, int whiten, double ridge, double* __restrict__ Adiag,
                       double* __restrict__ scal /* [0]=trace [1]=maxdiag */)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double tr = 0.0, mx = 0.0;
    for (int j = 0; j < d; ++j) {
        const double s = S[(size_t)j * d + j];
        tr = __dadd_rn(tr, s);
        if (s > mx) mx = s;
    }
    const double add = (whiten == FRR_RIDGE) ? __dmul_rn(ridge, __ddiv_rn(tr, (double)d)) : 0.0;
    for (int j = 0; j < d; ++j) Adiag[j] = __dadd_rn(S[(size_t)j * d + j], add);
    scal[0] = tr;
    scal[1] = mx;
}

// Column j of the unpivoted Cholesky factor, stored column-major: LT[k * d + i] = L_ik.
//   L_jj = sqrt(A_jj - sum_{k<j} L_jk^2),  L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj  (i > j).
// Every thread recomputes the pivot with the same operations, so all agree on it.
__global__ void k_chol_col(const double* __restrict__ S, const double* __restrict__ Adiag, int d, int j,
                           double tol_abs, double* __restrict__ LT, int* __restrict__ status)
{
    const int i = j + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double s = Adiag[j];
    double t = (i == j) ? 0.0 : S[(size_t)j * d + i];
    for (int k = 0; k < j; ++k) {
        const double ljk = LT[(size_t)k * d + j];
        s = __dsub_rn(s, __dmul_rn(ljk, ljk));
        if (i != j) t = __dsub_rn(t, __dmul_rn(LT[(size_t)k * d + i], ljk));
    }
    if (!(s > tol_abs)) {
        if (i == j) atomicExch(status, 1);
        return;
    }
    const double ljj = __dsqrt_rn(s);
    LT[(size_t)j * d + i] = (i == j) ? ljj : __ddiv_rn(t, ljj);
}

__global__ void k_diag_factor(const double* __restrict__ S, int d, double tol_abs, double* __restrict__ LT,
                              int* __restrict__ status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const double s = S[(size_t)j * d + j];
    if (!(s > tol_abs)) { atomicExch(status, 1); return; }
    LT[(size_t)j * d + j] = __dsqrt_rn(s);
}

// Row i of Zc solves L z = Xc_i^T by forward substitution (ascending k):
//   z_j = (Xc_ij - sum_{k<j} L_jk z_k) / L_jj.  ZT is column-major (ZT[j * n + i]).
__global__ void k_forward(const double* __restrict__ Xc, const double* __restrict__ LT, int n, int d,
                          double* __restrict__ ZT)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int j = 0; j < d; ++j) {
        double t = Xc[(size_t)i * d + j];
        for (int k = 0; k < j; ++k) t = __dsub_rn(t, __dmul_rn(LT[(size_t)k * d + j], ZT[(size_t)k * n + i]));
        ZT[(size_t)j * n + i] = __ddiv_rn(t, LT[(size_t)j * d + j]);
    }
}

__global__ void k_transpose(const double* __restrict__ ZT, int n, int d, double* __restrict__ Z)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * d) return;
    const int i = (int)(idx / d), j = (int)(idx % d);
    Z[idx] = ZT[(size_t)j * n + i];
}

// qexp_j such that |Zc_ij * 2^qexp_j| <= 2^kQBits for every i
__global__ void k_qexp(const double* __restrict__ Z, int n, int d, int* __restrict__ qexp)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(Z[(size_t)i * d + j]));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e with f in [0.5, 1): mx < 2^e
    qexp[j] = (mx > 0.0) ? (kQBits - e) : 0;
}

// K-order derived arrays (p = K position, u = unit at p).
__global__ void k_derive(const double* __restrict__ Z, int n, int d, int kpad, int dpad32,
                         const int* __restrict__ qexp, float* __restrict__ Z32, __nv_bfloat16* __restrict__ Zhi,
                         __nv_bfloat16* __restrict__ Zlo, long long* __restrict__ Q)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)kpad * dpad32) return;
    const int p = (int)(idx / dpad32), j = (int)(idx % dpad32);
    const int u = unit_of_kpos(p);
    const double z = (u < n && j < d) ? Z[(size_t)u * d + j] : 0.0;
    Z32[idx] = (float)z;
    if (j < d) {
        const __nv_bfloat16 hi = __double2bfloat16(z);
        const __nv_bfloat16 lo = __double2bfloat16(z - (double)__bfloat162float(hi));
        Zhi[(size_t)j * kpad + p] = hi;
        Zlo[(size_t)j * kpad + p] = lo;
        Q[(size_t)p * d + j] = llrint(ldexp(z, qexp[j]));
    }
}

__global__ void k_qsum(const long long* __restrict__ Q, int kpad, int d, long long* __restrict__ Qsum)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    long long s = 0;
    for (int p = 0; p < kpad; ++p) s += Q[(size_t)p * d + j];
    Qsum[j] = s;
}

// Per-column error terms of the bulk paths, bounding |s_hat_j - s_j| for the
// treated sum s_j = sum_{i in T} Zc_ij:
//   representation: sum_i |Zc_ij - repr(Zc_ij)|  (an exact bound for any treated set);
//   accumulation:   u * sum_p (|E T_p| + lambda sd(T_p) + |Zc_pj|), with T_p the
//     partial sum after K position p under complete randomization
//     (E T_p = (n1/n) sum_{p'<=p} Z, Var T_p <= pi(1-pi) n/(n-1) sum_{p'<=p} Z^2),
//     one rounding of relative size u per accumulated term.
// SIMT FP32: u = 2^-24 (round to nearest), one pass.
// Tensor cores: u = 2^-23 (truncation allowed), two passes (hi and lo terms).
__global__ void k_band_cols(const double* __restrict__ Z, int n, int d, int n1, int kused,
                            double* __restrict__ eps32, double* __restrict__ eps_tc)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const double pi = (double)n1 / n;
    const double vf = pi * (1.0 - pi) * (double)n / (double)(n - 1);
    double s1 = 0.0, s2 = 0.0, acc = 0.0, r32 = 0.0, rtc = 0.0;
    for (int p = 0; p < kused; ++p) {
        const int u = unit_of_kpos(p);
        if (u >= n) continue;
        const double z = Z[(size_t)u * d + j];
        s1 += z;
        s2 += z * z;
        acc += fabs(pi * s1) + kBandLambda * sqrt(vf * s2) + fabs(z);
        r32 += fabs(z - (double)(float)z);
        const double hi = (double)__bfloat162float(__double2bfloat16(z));
        const double lo = (double)__bfloat162float(__double2bfloat16(z - hi));
        rtc += fabs((z - hi) - lo);
    }
    eps32[j] = r32 + ldexp(acc, -24);
    eps_tc[j] = rtc + 2.0 * ldexp(acc, -23);
}

BandConsts band_from_eps(const std::vector<double>& eps, double c_M, int64_t d)
{
    double ss = 0.0;
    for (double e : eps) ss += e * e;
    const double en = sqrt(ss);
    const double u = ldexp(1.0, -24);
    const double g = (double)(d + 2) * u / (1.0 - (double)(d + 2) * u);
    BandConsts b;
    b.lin = 2.0 * sqrt(c_M) * en;
    b.quad = 3.0 * c_M * ss;
    b.rel = g;
    return b;
}

}  // namespace

frr_status prep_run(frr_ctx* ctx, const double* X_host)
{
    const int n = (int)ctx->n, d = (int)ctx->d;
    cudaStream_t s = ctx->stream;
    const size_t nd = (size_t)n * d;
    double *X = nullptr, *xbar = nullptr, *Xc = nullptr, *S = nullptr, *Adiag = nullptr, *LT = nullptr,
           *ZT = nullptr, *scal = nullptr, *eps = nullptr;
    int* status = nullptr;
    frr_status rc = FRR_OK;
    auto fail = [&](cudaError_t e) { ctx->failed = true; rc = (e == cudaErrorMemoryAllocation) ? FRR_E_NOMEM : FRR_E_CUDA; };
#define PREP_CHECK(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { fail(_e); goto cleanup; } } while (0)

    PREP_CHECK(cudaMalloc(&X, nd * sizeof(double)));
    PREP_CHECK(cudaMalloc(&xbar, d * sizeof(double)));
    PREP_CHECK(cudaMalloc(&Xc, nd * sizeof(double)));
    PREP_CHECK(cudaMalloc(&S, (size_t)d * d * sizeof(double)));
    PREP_CHECK(cudaMalloc(&Adiag, d * sizeof(double)));
    PREP_CHECK(cudaMalloc(&LT, (size_t)d * d * sizeof(double)));
    PREP_CHECK(cudaMalloc(&ZT, nd * sizeof(double)));
    PREP_CHECK(cudaMalloc(&scal, 4 * sizeof(double)));
    PREP_CHECK(cudaMalloc(&eps, 2 * (size_t)d * sizeof(double)));
    PREP_CHECK(cudaMalloc(&status, sizeof(int)));
    PREP_CHECK(cudaMemsetAsync(status, 0, sizeof(int), s));
    PREP_CHECK(cudaMemsetAsync(LT, 0, (size_t)d * d * sizeof(double), s));
    PREP_CHECK(cudaMemcpyAsync(X, X_host, nd * sizeof(double), cudaMemcpyHostToDevice, s));

    k_colmean<<<ceil_div(d, 128), 128, 0, s>>>(X, n, d, xbar);
    k_center<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(X, xbar, n, d, Xc);
    {
        dim3 blk(32, 8), grd(ceil_div(d, 32), ceil_div(d, 8));
        k_cov<<<grd, blk, 0, s>>>(Xc, n, d, S);
    }
    k_diag<<<1, 1, 0, s>>>(S, d, ctx->opts.whiten, ctx->opts.ridge, Adiag, scal);
    PREP_CHECK(cudaGetLastError());
    {
        double sc[2];
        PREP_CHECK(cudaMemcpyAsync(sc, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaStreamSynchronize(s));
        const double tol_abs = 1e-12 * sc[1];
        if (ctx->opts.whiten == FRR_DIAG) {
            k_diag_factor<<<ceil_div(d, 128), 128, 0, s>>>(S, d, tol_abs, LT, status);
        } else {
            for (int j = 0; j < d; ++j)
                k_chol_col<<<ceil_div(d - j, 128), 128, 0, s>>>(S, Adiag, d, j, tol_abs, LT, status);
        }
        PREP_CHECK(cudaGetLastError());
        int st = 0;
        PREP_CHECK(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaStreamSynchronize(s));
        if (st != 0) { rc = FRR_E_DEGENERATE; goto cleanup; }
    }
    k_forward<<<ceil_div(n, 32), 32, 0, s>>>(Xc, LT, n, d, ZT);
    k_transpose<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(ZT, n, d, ctx->Zc64);
    k_qexp<<<ceil_div(d, 128), 128, 0, s>>>(ctx->Zc64, n, d, ctx->qexp);
    {
        const size_t tot = (size_t)ctx->kpad * ctx->dpad32;
        PREP_CHECK(cudaMemsetAsync(ctx->Zhi, 0, (size_t)d * ctx->kpad * sizeof(__nv_bfloat16), s));
        PREP_CHECK(cudaMemsetAsync(ctx->Zlo, 0, (size_t)d * ctx->kpad * sizeof(__nv_bfloat16), s));
        k_derive<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->Zc64, n, d, ctx->kpad, ctx->dpad32, ctx->qexp,
                                                              ctx->Z32, ctx->Zhi, ctx->Zlo, ctx->Q);
    }
    k_qsum<<<ceil_div(d, 128), 128, 0, s>>>(ctx->Q, ctx->kpad, d, ctx->Qsum);
    k_band_cols<<<ceil_div(d, 128), 128, 0, s>>>(ctx->Zc64, n, d, (int)ctx->n1, ctx->kused, eps, eps + d);
    PREP_CHECK(cudaGetLastError());
    {
        std::vector<double> e32(d), etc(d);
        PREP_CHECK(cudaMemcpyAsync(e32.data(), eps, d * sizeof(double), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaMemcpyAsync(etc.data(), eps + d, d * sizeof(double), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaStreamSynchronize(s));
        ctx->band32 = band_from_eps(e32, ctx->c_M, d);
        ctx->band_tc = band_from_eps(etc, ctx->c_M, d);
    }
    {
        std::vector<uint64_t> tab(64 * 64);
        for (int c = 0; c < 64; ++c)
            for (int m = 0; m < 64; ++m) tab[c * 64 + m] = binom_host(c, m);
        PREP_CHECK(cudaMemcpyAsync(ctx->binom, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        PREP_CHECK(cudaStreamSynchronize(s));
    }

cleanup:
#undef PREP_CHECK
    cudaFree(X); cudaFree(xbar); cudaFree(Xc); cudaFree(S); cudaFree(Adiag); cudaFree(LT);
    cudaFree(ZT); cudaFree(scal); cudaFree(eps); cudaFree(status);
    return rc;
}

}  // namespace frr
