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



// ---- blocked factorisation with the same operation order --------------------------
// Panels of kP columns. Every entry of the working matrix receives its subtractions
// "- L_ik L_jk" (resp. "- L_jk z_ik") one by one in ascending k -- earlier panels through
// the trailing updates, the current panel inside the panel kernel -- followed by the
// same square root / division, so the results equal the column-by-column definition
// bit for bit while the work runs in parallel.
constexpr int kP = 32;

// The panel kernels work on groups of 32 rows with lane = row; the pw <= 32 panel columns are
// spread over kPW warps (warp w owns columns w, w + kPW, ...), so that the independent updates
// of a step run on several warps at once: B300 issues a warp's FP64 instructions about one per
// 64 cycles, so one warp per row group (all 32 columns in one thread) is issue-bound. Each
// step publishes the finished column through shared memory; the owner of the next column
// updates and finishes that column first (look-ahead), then the other owned columns follow.
constexpr int kPW = 8;
constexpr int kPC = kP / kPW;  // columns per warp

// RN(a / b) from y = RN(1 / b) by Markstein's method (P. Markstein, IBM J. Res. Dev. 34(1),
// 1990): from a quotient within one ulp of a / b, q + (a - b q) y rounded once (FMA, with the
// residual a - b q exact) is the correctly rounded quotient; one correction step from RN(a y)
// supplies such a quotient. The intermediate values must neither underflow nor overflow, so
// operands outside a safe exponent range (zero and subnormals included) use the division
// operator. Five dependent FP64 operations instead of a division.
__device__ __forceinline__ double div_rn_recip(double a, double b, double y)
{
    const int ea = (__double2hiint(a) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
    if (ea < 1023 - 900 || ea > 1023 + 900 || eb < 1023 - 400 || eb > 1023 + 400) return __ddiv_rn(a, b);
    const double q0 = __dmul_rn(a, y);
    const double r0 = __fma_rn(-q0, b, a);
    const double q1 = __fma_rn(r0, y, q0);
    const double r1 = __fma_rn(-q1, b, a);
    return __fma_rn(r1, y, q1);
}

// Right-looking elimination of one 32-row group (lane = row, t[c] = column w + kPW c) against a
// finished lower-triangular pw x pw block: for jj ascending, t_jj /= L_jj,jj, then
// t_kk -= L_kk,jj t_jj for jj < kk < pw. Every entry gets its subtractions in ascending jj and
// then its division, as in the column-by-column definition. Lc[jj][kk] = L_{kk,jj} (kk >= jj),
// Ld / Yd the diagonal and its reciprocals, Zs[jj][lane] the exchange of finished columns.
__device__ __forceinline__ void eliminate_rows(double (&t)[kPC], int pw, const double (*Lc)[kP + 1],
                                               const double* Ld, const double* Yd, double (*Zs)[32], int w, int lane)
{
    if (w == 0) {
        t[0] = div_rn_recip(t[0], Ld[0], Yd[0]);
        Zs[0][lane] = t[0];
    }
    for (int jj = 0; jj < pw; ++jj) {
        __syncthreads();
        const double z = Zs[jj][lane];
        const int nxt = jj + 1;
        if (nxt < pw && w == nxt % kPW) {
#pragma unroll
            for (int c = 0; c < kPC; ++c)
                if (w + kPW * c == nxt) {
                    t[c] = div_rn_recip(__dsub_rn(t[c], __dmul_rn(Lc[jj][nxt], z)), Ld[nxt], Yd[nxt]);
                    Zs[nxt][lane] = t[c];
                }
        }
#pragma unroll
        for (int c = 0; c < kPC; ++c) {
            const int kk = w + kPW * c;
            if (kk > nxt && kk < pw) t[c] = __dsub_rn(t[c], __dmul_rn(Lc[jj][kk], z));
        }
    }
}

// Panel [k0, k0 + pw) of the Cholesky factor, in place in A (row-major d x d, lower part:
// working values, final L on exit). Every CTA factors the pw x pw diagonal block (lane = row
// of the block) and then finishes its own 32 rows below it; CTA 0 writes the block back.
__global__ void __launch_bounds__(kP * kPW)
k_chol_panel(double* __restrict__ A, int d, int k0, int pw, const double* __restrict__ scal, int* __restrict__ status)
{
    const double tol_abs = __dmul_rn(1e-12, scal[1]);  // pivot tolerance relative to max S_jj
    __shared__ double Lc[kP][kP + 1];  // Lc[jj][r] = L_{k0+r, k0+jj}, r >= jj
    __shared__ double Zs[kP][32];
    __shared__ double Ld[kP], Yd[kP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double t[kPC];
    {
        // ---- diagonal block, right-looking: at step jj the pivot becomes L_jj,jj, the rows
        // below divide by it, and every later entry (kk, r) with jj < kk <= r subtracts
        // L_r,jj L_kk,jj (the diagonal entry subtracts a square)
        const int r = lane;
#pragma unroll
        for (int c = 0; c < kPC; ++c) {
            const int kk = w + kPW * c;
            t[c] = (r < pw && kk <= r) ? A[(size_t)(k0 + r) * d + k0 + kk] : 0.0;
        }
        // finish column j held in tc by its owner warp: pivot on lane j, division below it
        auto finish_col = [&](double& tc, int j) {
            double piv = 0.0;
            if (lane == j) {
                if (!(tc > tol_abs)) atomicExch(status, 1);
                piv = __dsqrt_rn(tc > 0.0 ? tc : 1.0);
                Ld[j] = piv;
            }
            piv = __shfl_sync(0xffffffffu, piv, j);
            if (lane == j) tc = piv;
            else if (lane > j && lane < pw) tc = __ddiv_rn(tc, piv);
            if (lane >= j && lane < pw) Lc[j][lane] = tc;
        };
        if (w == 0) finish_col(t[0], 0);
        for (int jj = 0; jj < pw; ++jj) {
            __syncthreads();
            const double lrj = (r >= jj && r < pw) ? Lc[jj][r] : 0.0;
            const int nxt = jj + 1;
            if (nxt < pw && w == nxt % kPW) {
#pragma unroll
                for (int c = 0; c < kPC; ++c)
                    if (w + kPW * c == nxt) {
                        if (r >= nxt && r < pw) t[c] = __dsub_rn(t[c], __dmul_rn(lrj, Lc[jj][nxt]));
                        finish_col(t[c], nxt);
                    }
            }
#pragma unroll
            for (int c = 0; c < kPC; ++c) {
                const int kk = w + kPW * c;
                if (kk > nxt && kk < pw && r >= kk && r < pw) t[c] = __dsub_rn(t[c], __dmul_rn(lrj, Lc[jj][kk]));
            }
        }
        if (blockIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < kPC; ++c) {
                const int kk = w + kPW * c;
                if (r < pw && kk <= r) A[(size_t)(k0 + r) * d + k0 + kk] = t[c];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < pw) Yd[threadIdx.x] = __ddiv_rn(1.0, Ld[threadIdx.x]);
    // ---- this CTA's 32 rows below the block
    const int r = k0 + pw + blockIdx.x * 32 + lane;
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
        const int kk = w + kPW * c;
        t[c] = (r < d && kk < pw) ? A[(size_t)r * d + k0 + kk] : 0.0;
    }
    __syncthreads();
    eliminate_rows(t, pw, Lc, Ld, Yd, Zs, w, lane);
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
        const int kk = w + kPW * c;
        if (r < d && kk < pw) A[(size_t)r * d + k0 + kk] = t[c];
    }
}

// Trailing update after panel [k0, k0 + pw): A_ij -= L_ik L_jk for k in the panel (ascending),
// for k0 + pw <= j <= i < d. 32 x 32 tiles, lower-triangle tiles only.
__global__ void __launch_bounds__(256)
k_chol_trailing(double* __restrict__ A, int d, int k0, int pw)
{
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    __shared__ double Li[32][kP + 1], Lj[32][kP + 1];
    const int base = k0 + pw;
    const int i0 = base + 32 * ti, j0 = base + 32 * tj;
    for (int e = threadIdx.x; e < 32 * kP; e += blockDim.x) {
        const int rr = e / kP, kk = e % kP;
        Li[rr][kk] = (i0 + rr < d && kk < pw) ? A[(size_t)(i0 + rr) * d + k0 + kk] : 0.0;
        Lj[rr][kk] = (j0 + rr < d && kk < pw) ? A[(size_t)(j0 + rr) * d + k0 + kk] : 0.0;
    }
    __syncthreads();
    const int jj = threadIdx.x & 31;
    for (int ii = threadIdx.x >> 5; ii < 32; ii += blockDim.x >> 5) {
        const int i = i0 + ii, j = j0 + jj;
        if (i >= d || j > i) continue;
        double v = A[(size_t)i * d + j];
        for (int kk = 0; kk < pw; ++kk) v = __dsub_rn(v, __dmul_rn(Li[ii][kk], Lj[jj][kk]));
        A[(size_t)i * d + j] = v;
    }
}

// Panel [k0, k0 + pw) of the forward substitution Zc = Xc L^{-T}, in place in T (n x d
// row-major: working values, final Zc on exit): 32 rows per CTA, eliminated against the
// panel's diagonal block of L (z_ij = (t_ij - sum_{k<j} L_jk z_ik) / L_jj, subtractions in
// ascending k).
__global__ void __launch_bounds__(kP * kPW)
k_fwd_panel(double* __restrict__ T, const double* __restrict__ L, int n, int d, int k0, int pw)
{
    __shared__ double Lc[kP][kP + 1];  // Lc[jj][kk] = L_{k0+kk, k0+jj}, kk >= jj
    __shared__ double Zs[kP][32];
    __shared__ double Ld[kP], Yd[kP];
    for (int e = threadIdx.x; e < kP * kP; e += blockDim.x) {
        const int jj = e / kP, kk = e % kP;
        Lc[jj][kk] = (kk < pw && kk >= jj) ? L[(size_t)(k0 + kk) * d + k0 + jj] : 0.0;
    }
    if (threadIdx.x < pw) {
        const double l = L[(size_t)(k0 + threadIdx.x) * d + k0 + threadIdx.x];
        Ld[threadIdx.x] = l;
        Yd[threadIdx.x] = __ddiv_rn(1.0, l);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    double t[kPC];
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
        const int kk = w + kPW * c;
        t[c] = (i < n && kk < pw) ? T[(size_t)i * d + k0 + kk] : 0.0;
    }
    __syncthreads();
    eliminate_rows(t, pw, Lc, Ld, Yd, Zs, w, lane);
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
        const int kk = w + kPW * c;
        if (i < n && kk < pw) T[(size_t)i * d + k0 + kk] = t[c];
    }
}

// T_ij -= L_jk z_ik for k in panel [k0, k0 + pw) (ascending), j >= k0 + pw. 32 x 32 tiles.
__global__ void __launch_bounds__(256)
k_fwd_trailing(double* __restrict__ T, const double* __restrict__ L, int n, int d, int k0, int pw)
{
    __shared__ double Zi[32][kP + 1], Lj[32][kP + 1];
    const int i0 = 32 * blockIdx.y, j0 = k0 + pw + 32 * blockIdx.x;
    for (int e = threadIdx.x; e < 32 * kP; e += blockDim.x) {
        const int rr = e / kP, kk = e % kP;
        Zi[rr][kk] = (i0 + rr < n && kk < pw) ? T[(size_t)(i0 + rr) * d + k0 + kk] : 0.0;
        Lj[rr][kk] = (j0 + rr < d && kk < pw) ? L[(size_t)(j0 + rr) * d + k0 + kk] : 0.0;
    }
    __syncthreads();
    const int jj = threadIdx.x & 31;
    for (int ii = threadIdx.x >> 5; ii < 32; ii += blockDim.x >> 5) {
        const int i = i0 + ii, j = j0 + jj;
        if (i >= n || j >= d) continue;
        double v = T[(size_t)i * d + j];
        for (int kk = 0; kk < pw; ++kk) v = __dsub_rn(v, __dmul_rn(Lj[jj][kk], Zi[ii][kk]));
        T[(size_t)i * d + j] = v;
    }
}

// A = S with the ridge on the diagonal (lower part is what the factorisation reads)
__global__ void k_init_A(const double* __restrict__ S, const double* __restrict__ Adiag, int d, double* __restrict__ A)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)d * d) return;
    const int i = (int)(idx / d), j = (int)(idx % d);
    A[idx] = (i == j) ? Adiag[i] : S[idx];
}

// diagonal whitening: L = diag(sqrt(S_jj)) stored row-major (zero elsewhere)
__global__ void k_diag_L(const double* __restrict__ S, int d, const double* __restrict__ scal, double* __restrict__ A,
                         int* status)
{
    const double tol_abs = __dmul_rn(1e-12, scal[1]);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)d * d) return;
    const int i = (int)(idx / d), j = (int)(idx % d);
    if (i != j) { A[idx] = 0.0; return; }
    const double s = S[idx];
    if (!(s > tol_abs)) atomicExch(status, 1);
    A[idx] = __dsqrt_rn(s > 0.0 ? s : 1.0);
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

// Balanced base-256 digits of Q: Q = sum_{k<7} q_k 256^k with q_k in [-128, 127], plane k
// stored K-major as BF16 (integers of this size are exact): Zq[(k d + j) kpad + p].
__global__ void k_digits(const long long* __restrict__ Q, int kpad, int d, __nv_bfloat16* __restrict__ Zq)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)kpad * d) return;
    const int j = (int)(idx / kpad), p = (int)(idx % kpad);
    long long v = Q[(size_t)p * d + j];
    for (int k = 0; k < 7; ++k) {
        int q = (int)(v & 0xFF);
        if (q >= 128) q -= 256;
        v = (v - q) >> 8;
        Zq[((size_t)k * d + j) * kpad + p] = __float2bfloat16_rn((float)q);
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
__global__ void __launch_bounds__(256)
k_band_cols(const double* __restrict__ Z, int n, int d, int n1, int kused, double* __restrict__ eps32,
            double* __restrict__ eps_tc)
{
    // one CTA per column; thread t covers K positions [t * per, (t + 1) * per)
    __shared__ double ws1[8], ws2[8], wacc[8], wr32[8], wrtc[8];
    const int j = blockIdx.x;
    const int per = (kused + 255) / 256;
    const int p0 = threadIdx.x * per;
    const double pi = (double)n1 / n;
    const double vf = pi * (1.0 - pi) * (double)n / (double)(n - 1);
    double l1 = 0.0, l2 = 0.0;
    for (int p = p0; p < p0 + per && p < kused; ++p) {
        const int u = unit_of_kpos(p);
        if (u < n) {
            const double z = Z[(size_t)u * d + j];
            l1 += z;
            l2 += z * z;
        }
    }
    // exclusive prefix of (l1, l2) over threads
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double i1 = l1, i2 = l2;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double y1 = __shfl_up_sync(kFull, i1, off), y2 = __shfl_up_sync(kFull, i2, off);
        if (lane >= off) { i1 += y1; i2 += y2; }
    }
    if (lane == 31) { ws1[warp] = i1; ws2[warp] = i2; }
    __syncthreads();
    double b1 = 0.0, b2 = 0.0;
    for (int w = 0; w < warp; ++w) { b1 += ws1[w]; b2 += ws2[w]; }
    double s1 = b1 + i1 - l1, s2 = b2 + i2 - l2;
    double acc = 0.0, r32 = 0.0, rtc = 0.0;
    for (int p = p0; p < p0 + per && p < kused; ++p) {
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
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        acc += __shfl_xor_sync(kFull, acc, off);
        r32 += __shfl_xor_sync(kFull, r32, off);
        rtc += __shfl_xor_sync(kFull, rtc, off);
    }
    if (lane == 0) { wacc[warp] = acc; wr32[warp] = r32; wrtc[warp] = rtc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, R32 = 0.0, RTC = 0.0;
        for (int w = 0; w < 8; ++w) { A += wacc[w]; R32 += wr32[w]; RTC += wrtc[w]; }
        eps32[j] = R32 + ldexp(A, -24);
        eps_tc[j] = RTC + 2.0 * ldexp(A, -23);
    }
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

// C(c, m) for c, m < 64 at [c * 64 + m] (Pascal's rule; every entry fits in 64 bits), built once
const uint64_t* binom_table()
{
    static const std::vector<uint64_t> tab = [] {
        std::vector<uint64_t> t(64 * 64, 0);
        for (int c = 0; c < 64; ++c) {
            t[(size_t)c * 64] = 1;
            for (int m = 1; m <= c; ++m) t[(size_t)c * 64 + m] = t[(size_t)(c - 1) * 64 + m - 1] + t[(size_t)(c - 1) * 64 + m];
        }
        return t;
    }();
    return tab.data();
}

frr_status prep_run(frr_ctx* ctx, const double* X_host)
{
    const int n = (int)ctx->n, d = (int)ctx->d;
    cudaStream_t s = ctx->stream;
    const size_t nd = (size_t)n * d;
    double *X = nullptr, *xbar = nullptr, *Xc = nullptr, *S = nullptr, *Adiag = nullptr, *Lm = nullptr,
           *ZT = nullptr, *scal = nullptr, *eps = nullptr;
    int* status = nullptr;
    frr_status rc = FRR_OK;
    auto fail = [&](cudaError_t e) { ctx->failed = true; rc = (e == cudaErrorMemoryAllocation) ? FRR_E_NOMEM : FRR_E_CUDA; };
#define PREP_CHECK(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { fail(_e); goto cleanup; } } while (0)

    cudaMemPool_t pool = temp_pool(ctx->device);
    if (pool == nullptr) return FRR_E_CUDA;
    PREP_CHECK(cudaMallocFromPoolAsync(&X, nd * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&xbar, d * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&Xc, nd * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&S, (size_t)d * d * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&Adiag, d * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&Lm, (size_t)d * d * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&ZT, nd * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&scal, 4 * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&eps, 2 * (size_t)d * sizeof(double), pool, s));
    PREP_CHECK(cudaMallocFromPoolAsync(&status, sizeof(int), pool, s));
    PREP_CHECK(cudaMemsetAsync(status, 0, sizeof(int), s));
    PREP_CHECK(cudaMemsetAsync(Lm, 0, (size_t)d * d * sizeof(double), s));
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
        // The pivot tolerance is read on the device (scal[1] = max S_jj), and a failed pivot is
        // only flagged (the factorisation goes on with a unit pivot, so every later value stays
        // finite): the host learns both at the single synchronisation at the end.
        const size_t dd = (size_t)d * d;
        // forward substitution in place on a copy of Xc (ZT holds n x d row-major here)
        PREP_CHECK(cudaMemcpyAsync(ZT, Xc, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (ctx->opts.whiten == FRR_DIAG) {
            k_diag_L<<<(unsigned)((dd + 255) / 256), 256, 0, s>>>(S, d, scal, Lm, status);
            for (int k0 = 0; k0 < d; k0 += kP) {
                const int pw = (d - k0) < kP ? (d - k0) : kP;
                k_fwd_panel<<<ceil_div(n, 32), kP * kPW, 0, s>>>(ZT, Lm, n, d, k0, pw);
                const int right = d - k0 - pw;
                if (right > 0)
                    k_fwd_trailing<<<dim3(ceil_div(right, 32), ceil_div(n, 32)), 256, 0, s>>>(ZT, Lm, n, d, k0, pw);
            }
        } else {
            // Both factorisations are chains of latency-bound panels. Step p of the forward
            // substitution needs only column panel p of L, which is final once Cholesky panel
            // p is done (later trailing updates touch columns to its right), so it runs on a
            // second stream, one panel behind: the two chains overlap.
            k_init_A<<<(unsigned)((dd + 255) / 256), 256, 0, s>>>(S, Adiag, d, Lm);
            const int np = ceil_div(d, kP);
            std::vector<cudaEvent_t> evs((size_t)np + 2, nullptr);
            for (auto& e : evs) PREP_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            PREP_CHECK(cudaEventRecord(evs[np], s));
            PREP_CHECK(cudaStreamWaitEvent(ctx->aux, evs[np], 0));
            for (int p = 0, k0 = 0; k0 < d; ++p, k0 += kP) {
                const int pw = (d - k0) < kP ? (d - k0) : kP;
                const int below = d - k0 - pw;
                k_chol_panel<<<below > 0 ? ceil_div(below, 32) : 1, kP * kPW, 0, s>>>(Lm, d, k0, pw, scal, status);
                PREP_CHECK(cudaEventRecord(evs[p], s));
                PREP_CHECK(cudaStreamWaitEvent(ctx->aux, evs[p], 0));
                k_fwd_panel<<<ceil_div(n, 32), kP * kPW, 0, ctx->aux>>>(ZT, Lm, n, d, k0, pw);
                if (below > 0) {
                    const int tiles = ceil_div(below, 32);
                    k_chol_trailing<<<dim3(tiles, tiles), 256, 0, s>>>(Lm, d, k0, pw);
                    k_fwd_trailing<<<dim3(ceil_div(below, 32), ceil_div(n, 32)), 256, 0, ctx->aux>>>(ZT, Lm, n, d, k0,
                                                                                                  pw);
                }
            }
            PREP_CHECK(cudaEventRecord(evs[np + 1], ctx->aux));
            PREP_CHECK(cudaStreamWaitEvent(s, evs[np + 1], 0));
            for (auto& e : evs) cudaEventDestroy(e);
        }
        PREP_CHECK(cudaGetLastError());
    }
    PREP_CHECK(cudaMemcpyAsync(ctx->Zc64, ZT, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_qexp<<<ceil_div(d, 128), 128, 0, s>>>(ctx->Zc64, n, d, ctx->qexp);
    {
        const size_t tot = (size_t)ctx->kpad * ctx->dpad32;
        PREP_CHECK(cudaMemsetAsync(ctx->Zhi, 0, (size_t)d * ctx->kpad * sizeof(__nv_bfloat16), s));
        PREP_CHECK(cudaMemsetAsync(ctx->Zlo, 0, (size_t)d * ctx->kpad * sizeof(__nv_bfloat16), s));
        k_derive<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->Zc64, n, d, ctx->kpad, ctx->dpad32, ctx->qexp,
                                                              ctx->Z32, ctx->Zhi, ctx->Zlo, ctx->Q);
    }
    k_qsum<<<ceil_div(d, 128), 128, 0, s>>>(ctx->Q, ctx->kpad, d, ctx->Qsum);
    k_digits<<<(unsigned)(((size_t)ctx->kpad * d + 255) / 256), 256, 0, s>>>(ctx->Q, ctx->kpad, d, ctx->Zq);
    k_band_cols<<<d, 256, 0, s>>>(ctx->Zc64, n, d, (int)ctx->n1, ctx->kused, eps, eps + d);
    PREP_CHECK(cudaGetLastError());
    // binomial table for exact enumeration (only shapes that allow it read it); the host
    // table is static, so the copy needs no synchronisation
    if (n <= kExactMaxN)
        PREP_CHECK(cudaMemcpyAsync(ctx->binom, binom_table(), 64 * 64 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    {
        // the single synchronisation of the preparation: pivot status and band inputs
        std::vector<double> e32(d), etc(d);
        int st = 0;
        PREP_CHECK(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaMemcpyAsync(e32.data(), eps, d * sizeof(double), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaMemcpyAsync(etc.data(), eps + d, d * sizeof(double), cudaMemcpyDeviceToHost, s));
        PREP_CHECK(cudaStreamSynchronize(s));
        if (st != 0) { rc = FRR_E_DEGENERATE; goto cleanup; }
        ctx->band32 = band_from_eps(e32, ctx->c_M, d);
        ctx->band_tc = band_from_eps(etc, ctx->c_M, d);
    }

cleanup:
#undef PREP_CHECK
    // stream-ordered release: no device-wide synchronisation
    for (void* p : {(void*)X, (void*)xbar, (void*)Xc, (void*)S, (void*)Adiag, (void*)Lm, (void*)ZT, (void*)scal,
                    (void*)eps, (void*)status})
        if (p) cudaFreeAsync(p, s);
    return rc;
}

}  // namespace frr
