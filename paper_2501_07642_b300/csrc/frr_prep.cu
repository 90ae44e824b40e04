// frr_prep.cu -- FP64 preparation of experiments on the GPU (frr_init, frr_batch_run).
//
// Sec. 2.2 works with covariates that are centred and whitened so that the
// Mahalanobis distance is Euclidean (App. A, remark on general Sigma_X):
//   xbar = column means, Xc = X - 1 xbar^T, S = Xc^T Xc / (n - 1),
//   S_lambda = S (+ ridge * tr(S)/d * I), S_lambda = L L^T, Zc = Xc L^{-T}.
// Every step uses explicitly rounded FP64 operations in ascending index order,
// one dependent chain per output, so the results do not depend on the launch
// shape; each term of a dot product (covariance, Cholesky factor, forward
// substitution) is added by one fused multiply-add (one rounding per term).
//
// From Zc (natural unit order) the kernels below derive the arrays the
// balance path reads, all in K-order (see frr_gen.cuh):
//   Z32  : FP32 copy for the SIMT path,
//   Zhi, Zlo : BF16 hi/lo split (Zc ~ hi + lo) for the tensor-core path,
//   Q    : fixed-point Zc * 2^qexp_j (int64) for the exact-sum recheck,
//   band : per-column error-band terms of both bulk paths.
//
// Any number of experiments of different shapes is prepared together: each kernel
// launch covers the blocks of every experiment (a table of experiment descriptors and,
// per launch, the prefix sums of their block counts), so a batch costs about as many
// launches as one experiment and its many small, latency-bound steps share the SMs.
#include "frr_internal.cuh"
#include "frr_gen.cuh"
#include "frr_tc_ptx.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace frr {

// One experiment's preparation as the kernels see it (device pointers).
struct PrepJob {
    int n, d, n1, whiten, kpad, dpad32, kused;
    int tc;  // covariance and cross-block forward-substitution updates from digit products on the tensor
             // cores (else the FP64 chains below)
    double ridge;
    // temporaries
    double *X, *xbar, *Xc, *S, *Adiag, *Lm, *ZT, *scal, *eps;
    long long* facc;  // forward-substitution sums of the tensor-core updates (n x d), or null
    int* status;
    // outputs (the context's arrays)
    double* Zc64;
    float* Z32;
    __nv_bfloat16 *Zhi, *Zlo;
    __half* Zq;
    long long *Q, *Qsum;
    int* qexp;
};

namespace {

#define PJ_ARGS const PrepJob* __restrict__ jobs, const unsigned* __restrict__ prefix, int E

// Status bits of a preparation: 1 = non-positive Cholesky pivot, 2 = a bounded wait expired,
// 4 = a non-finite covariate (found where the centring reads X).
constexpr int kStatusPivot = 1, kStatusTimeout = 2, kStatusNonFinite = 4;

// The job owning this block and the block's index within the job: prefix[e] is the first
// block of job e (jobs with no blocks have prefix[e] == prefix[e + 1]).
__device__ __forceinline__ const PrepJob& job_of(PJ_ARGS, unsigned& local)
{
    const unsigned b = blockIdx.x;
    int lo = 0, hi = E;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid;
    }
    local = b - prefix[lo];
    return jobs[lo];
}

// Column means: one chain of FP64 additions per column in ascending i, as the definition.
// The chain (64 cycles per dependent addition) sets the time, so its operands come from
// shared memory: warps 1..7 copy tiles of kCmRows rows x 32 columns (double-buffered) while
// warp 0, lane = column, adds the previous tile.
constexpr int kCmRows = 64;

__global__ void __launch_bounds__(256) k_colmean(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d;
    const int j0 = (int)lb * 32;
    __shared__ double tile[2][kCmRows][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (J.tc) {
        // tensor-core mode (the oracle's chain is not kept): eight row groups sum their rows
        // (lane = column) and the eight partial sums are added in order, a blocked sum with a
        // chain of n / 8 additions instead of n
        double sg = 0.0;
        if (j0 + lane < d)
            for (int i = w; i < n; i += 8) sg = __dadd_rn(sg, J.X[(size_t)i * d + j0 + lane]);
        tile[0][w][lane] = sg;
        __syncthreads();
        if (w == 0 && j0 + lane < d) {
            double t = tile[0][0][lane];
            for (int g = 1; g < 8; ++g) t = __dadd_rn(t, tile[0][g][lane]);
            J.xbar[j0 + lane] = __ddiv_rn(t, (double)n);
        }
        return;
    }
    const int ntiles = (n + kCmRows - 1) / kCmRows;
    auto load = [&](int t, int buf) {
        for (int r = w - 1; r < kCmRows; r += 7) {
            const int i = t * kCmRows + r, j = j0 + lane;
            tile[buf][r][lane] = (i < n && j < d) ? J.X[(size_t)i * d + j] : 0.0;
        }
    };
    if (w > 0) load(0, 0);
    __syncthreads();
    double s = 0.0;
    for (int t = 0; t < ntiles; ++t) {
        if (w > 0) {
            if (t + 1 < ntiles) load(t + 1, (t + 1) & 1);
        } else {
            const int rows = min(kCmRows, n - t * kCmRows);
            for (int r = 0; r < rows; ++r) s = __dadd_rn(s, tile[t & 1][r][lane]);
        }
        __syncthreads();
    }
    if (w == 0 && j0 + lane < d) J.xbar[j0 + lane] = __ddiv_rn(s, (double)n);
}

__global__ void k_center(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const size_t idx = (size_t)lb * blockDim.x + threadIdx.x;
    if (idx >= (size_t)J.n * J.d) return;
    const double x = J.X[idx];
    // every covariate passes here once: an all-ones exponent field (infinity or NaN) is
    // reported in the status word (integer instructions; the atomic only when one is found)
    if ((__double_as_longlong(x) & 0x7ff0000000000000ll) == 0x7ff0000000000000ll) atomicOr(J.status, kStatusNonFinite);
    const double v = __dsub_rn(x, J.xbar[idx % J.d]);
    J.Xc[idx] = v;
    J.ZT[idx] = v;  // the forward substitution works in place on a copy of Xc
    if (J.facc) J.facc[idx] = 0ll;
}

// S_jk = sum_i Xc_ij Xc_ik / (n - 1) for k >= j, mirrored (the product is commutative,
// so both halves are the value a separate (k, j) computation would give). 32 x 8 threads
// per block, blocks row-major over (ceil(d / 32), ceil(d / 8)).
__global__ void k_cov(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d;
    const unsigned gx = (unsigned)((d + 31) / 32);
    const int k = (int)(lb % gx) * 32 + threadIdx.x;
    const int j = (int)(lb / gx) * 8 + threadIdx.y;
    if (j >= d || k >= d || k < j) return;
    const double* Xc = J.Xc;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = __fma_rn(Xc[(size_t)i * d + j], Xc[(size_t)i * d + k], s);
    const double v = __ddiv_rn(s, (double)(n - 1));
    J.S[(size_t)j * d + k] = v;
    J.S[(size_t)k * d + j] = v;
}

// trace, max diagonal, and the diagonal of S_lambda (ridge added); one block per job. The
// trace is one chain of FP64 additions in ascending j (as the definition); the maximum (of
// non-negative values: an integer maximum of their bit patterns) and the ridge diagonal are
// spread over the block.
__global__ void __launch_bounds__(256) k_diag(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d;
    const double* S = J.S;
    __shared__ double s_tr;
    __shared__ unsigned long long s_mx[8];
    unsigned long long mx = 0ull;  // bits of +0.0
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(S[(size_t)j * d + j]);
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, mx, off);
        mx = o > mx ? o : mx;
    }
    if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
    if (J.tc) {
        // tensor-core mode (the oracle's chain is not kept): the trace as a blocked sum, each
        // thread's strided terms, then a tree in the warp, then the warps' sums in order
        __shared__ double s_part[8];
        double pt = 0.0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) pt = __dadd_rn(pt, S[(size_t)j * d + j]);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) pt = __dadd_rn(pt, __shfl_xor_sync(kFull, pt, off));
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = pt;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = s_part[0];
            for (int g = 1; g < (int)(blockDim.x >> 5); ++g) tr = __dadd_rn(tr, s_part[g]);
            s_tr = tr;
        }
    } else if (threadIdx.x == 0) {
        double tr = 0.0;
        int j = 0;
        for (; j + 8 <= d; j += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = S[(size_t)(j + u) * d + (j + u)];
#pragma unroll
            for (int u = 0; u < 8; ++u) tr = __dadd_rn(tr, v[u]);
        }
        for (; j < d; ++j) tr = __dadd_rn(tr, S[(size_t)j * d + j]);
        s_tr = tr;
    }
    __syncthreads();
    const double tr = s_tr;
    const double add = (J.whiten == FRR_RIDGE) ? __dmul_rn(J.ridge, __ddiv_rn(tr, (double)d)) : 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) J.Adiag[j] = __dadd_rn(S[(size_t)j * d + j], add);
    if (threadIdx.x == 0) {
        unsigned long long m = s_mx[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = s_mx[w] > m ? s_mx[w] : m;
        J.scal[0] = tr;
        J.scal[1] = __longlong_as_double((long long)m);
    }
}

// Working matrix of the factorisation: A = S with the ridge on the diagonal (the lower part
// is what the factorisation reads), or for diagonal whitening L = diag(sqrt(S_jj)) itself.
__global__ void k_init_L(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d;
    const size_t idx = (size_t)lb * blockDim.x + threadIdx.x;
    if (idx >= (size_t)d * d) return;
    const int i = (int)(idx / d), j = (int)(idx % d);
    if (J.whiten != FRR_DIAG) {
        J.Lm[idx] = (i == j) ? J.Adiag[i] : J.S[idx];
        return;
    }
    if (i != j) { J.Lm[idx] = 0.0; return; }
    const double tol_abs = __dmul_rn(1e-12, J.scal[1]);  // pivot tolerance relative to max S_jj
    const double s = J.S[idx];
    if (!(s > tol_abs)) atomicOr(J.status, kStatusPivot);
    J.Lm[idx] = __dsqrt_rn(s > 0.0 ? s : 1.0);
}

// ---- blocked factorisation with the same operation order --------------------------
// Panels of kP columns. Every entry of the working matrix receives its fused
// multiply-subtractions "- L_ik L_jk" (resp. "- L_jk z_ik") one by one in ascending k -- earlier panels through
// the trailing updates, the current panel inside the panel kernel -- followed by the
// same square root / division, so the results equal the column-by-column definition
// bit for bit while the work runs in parallel.
constexpr int kP = 32;

// The panel kernels work on groups of 32 rows with lane = row, one warp per panel column
// (kP warps). B300 runs FP64 at about one warp instruction per 19 cycles per SM, shared
// among the warps that issue it, and at most one per 64 cycles for a single warp; every
// issued FP64 instruction counts, predicated off or not. So the kernels let a column's
// dependent chain (its last update, then the square root or division) compete with as few
// other FP64 instructions as possible: warp w owns column w, applies the updates from
// columns jj < w as soon as each of them is published (one mbarrier per column, 32 lane
// arrivals after the lane's store of the finished value), finishes its column and stops.
// No block-wide barrier holds the warps in lockstep, and finished warps issue nothing.
constexpr int kPW = kP;  // warps per panel block

// Bounded wait for the publication of one column (phase `parity` of its mbarrier). On expiry
// the block's abort flag and the timeout bit are raised; later waits of the block return at once.
__device__ __forceinline__ bool wait_col(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status)
{
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = clock64();
    for (;;) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > tc::kWaitCycles) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

// Shared state of a panel block: the published columns Zs[jj][lane] with their mbarriers.
struct PanelSync {
    double Zs[kP][32];
    uint64_t bar[kP];
    int abort_flag;
};

__device__ __forceinline__ void panel_sync_init(PanelSync& ps)
{
    if (threadIdx.x < kP) tc::mbar_init(&ps.bar[threadIdx.x], 32);
    if (threadIdx.x == 0) ps.abort_flag = 0;
}

// Publish the finished value of column w for this lane's row (every lane of the warp arrives).
__device__ __forceinline__ void publish(PanelSync& ps, int w, int lane, double v)
{
    ps.Zs[w][lane] = v;
    tc::mbar_arrive(&ps.bar[w]);
}

// 1/sqrt(a) for a > 0 (normal or subnormal), within about half an ulp: a = m 4^h with m in
// [1, 4) (an even power of two split off in the exponent field); an FP32 seed y0 ~ 1/sqrt(m)
// to ~21 bits (the PTX reciprocal-square-root approximation of m's top 20 fraction bits), then
// one third-order step from the series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ... with
// e = 1 - m y0^2 (y0^2 is exact: y0 has 24 significant bits), y = y0 + y0 e (1/2 + 3e/8);
// the truncated terms are below 2^-59 relative. The seed moves between FP64 and FP32 by
// integer bit operations, not conversion instructions, so the dependent chain holds four
// FP64 operations (a column of the diagonal panel waits for it).
__device__ __forceinline__ double rsqrt_near(double a)
{
    long long bits = __double_as_longlong(a);
    int shift = 0;                      // a = m 2^(2 shift) with m in [1, 4)
    if ((bits >> 52) == 0) {            // subnormal: make it normal first (exact)
        a = __dmul_rn(a, 0x1p+64);
        bits = __double_as_longlong(a);
        shift -= 32;
    }
    const int h = ((int)(bits >> 52) - 1023) >> 1;  // floor of half the exponent
    const double m = __longlong_as_double(bits - ((long long)(2 * h) << 52));
    shift += h;
    // exponent field of m: 1023 or 1024 -> FP32 exponent field 127 or 128 (1023 - 127 = 896);
    // the top 20 fraction bits move along (the 32-bit arithmetic wraps harmlessly)
    const uint32_t hi = (uint32_t)__double2hiint(m);
    const float mf = __uint_as_float((hi << 3) - (896u << 23));
    float y32;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y32) : "f"(mf));
    const uint32_t fb = __float_as_uint(y32);  // y32 in (1/2, 1]: exact as a double
    const double y0 = __hiloint2double((int)((fb >> 3) + (896u << 20)), (int)(fb << 29));
    const double e = __fma_rn(-m, __dmul_rn(y0, y0), 1.0);
    const double y = __fma_rn(__dmul_rn(y0, e), __fma_rn(e, 0.375, 0.5), y0);
    // 1/sqrt(a) = y 2^-shift (exact scaling: the exponent of y stays in range)
    return __longlong_as_double(__double_as_longlong(y) - ((long long)shift << 52));
}

// RN(a / b) from y = RN(1 / b) by Markstein's method (P. Markstein, IBM J. Res. Dev. 34(1),
// 1990): from a quotient within one ulp of a / b, q + (a - b q) y rounded once (FMA, with the
// residual a - b q exact) is the correctly rounded quotient; one correction step from RN(a y)
// supplies such a quotient. Five dependent FP64 operations instead of a division. The
// intermediate values must neither underflow nor overflow, and a zero dividend must keep its
// sign, so the result is correct only when markstein_unsafe(a, b) is false.
__device__ __forceinline__ double div_markstein(double a, double b, double y)
{
    const double q0 = __dmul_rn(a, y);
    const double r0 = __fma_rn(-q0, b, a);
    const double q1 = __fma_rn(r0, y, q0);
    const double r1 = __fma_rn(-q1, b, a);
    return __fma_rn(r1, y, q1);
}

// Operands outside the safe exponent range of div_markstein (zero and subnormals included).
__device__ __forceinline__ bool markstein_unsafe(double a, double b)
{
    const int ea = (__double2hiint(a) >> 20) & 0x7ff, eb = (__double2hiint(b) >> 20) & 0x7ff;
    return ea < 1023 - 900 || ea > 1023 + 900 || eb < 1023 - 400 || eb > 1023 + 400;
}

// Column w of one 32-row group (lane = row, t = the working value) eliminated against a
// finished lower-triangular pw x pw block: t -= L_w,jj z_jj for jj < w ascending, as each
// z_jj is published (mbarrier phase `parity`), then t /= L_w,w; the result is published as
// column w. Lc[jj][kk] = L_{kk,jj} (kk >= jj), Ld / Yd the diagonal and its reciprocals.
// kExact = false divides by div_markstein and ORs markstein_unsafe into `unsafe` for rows
// that exist (row_ok; padding rows hold zeros and are never stored, and a zero dividend would
// otherwise send the last row block of every launch down the slow path); kExact = true uses
// the division operator.
template <bool kExact>
__device__ __forceinline__ double eliminate_col(double t, int w, int lane, const double (*Lc)[kP + 1],
                                                const double* Ld, const double* Yd, PanelSync& ps, uint32_t parity,
                                                bool row_ok, bool& unsafe, int* status, bool fast)
{
    for (int jj = 0; jj < w; ++jj) {
        if (!wait_col(&ps.bar[jj], parity, &ps.abort_flag, status)) break;
        t = __fma_rn(-Lc[jj][w], ps.Zs[jj][lane], t);
    }
    if (kExact) {
        t = __ddiv_rn(t, Ld[w]);
    } else if (fast) {
        t = __dmul_rn(t, Yd[w]);  // tensor-core mode: times the reciprocal, within 1.5 ulp of the quotient
    } else {
        unsafe |= row_ok && markstein_unsafe(t, Ld[w]);
        t = div_markstein(t, Ld[w], Yd[w]);
    }
    publish(ps, w, lane, t);
    return t;
}

// The row-panel elimination of a block: the fast pass with div_markstein, and, if any
// division of the block had operands outside its safe range (rare: zero or extreme values),
// the whole pass again from the original values with the division operator (the second
// phase of every column's mbarrier). Every warp of the block calls this (warps w >= pw only
// take part in the block-wide vote).
__device__ __forceinline__ double eliminate_panel_rows(double t0, int pw, int w, int lane, const double (*Lc)[kP + 1],
                                                       const double* Ld, const double* Yd, PanelSync& ps, bool row_ok,
                                                       int* status, bool fast)
{
    bool unsafe = false;
    double t = t0;
    if (w < pw) t = eliminate_col<false>(t0, w, lane, Lc, Ld, Yd, ps, 0u, row_ok, unsafe, status, fast);
    if (__syncthreads_or(unsafe) && w < pw)
        t = eliminate_col<true>(t0, w, lane, Lc, Ld, Yd, ps, 1u, row_ok, unsafe, status, fast);
    return t;
}

// Diagonal block of panel p (columns [32 p, 32 p + pw)) of the Cholesky factor, in place in
// Lm (row-major d x d, lower part: working values, final L on exit); one block per job, lane =
// row of the block, warp w = column w. Column w receives - L_r,jj L_w,jj for jj < w in
// ascending jj (each as soon as column jj is published), then its pivot L_w,w = sqrt(t_w,w)
// and the divisions of the rows below it. The rows below the block follow in k_chol_below,
// which reads the finished block (a separate launch: blocks of one launch may start after
// others have finished, so the block must not be overwritten while other blocks may still
// read it).
__global__ void __launch_bounds__(kP * kPW) k_chol_diag(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    double* __restrict__ A = J.Lm;
    const double tol_abs = __dmul_rn(1e-12, J.scal[1]);  // pivot tolerance relative to max S_jj
    __shared__ PanelSync ps;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = lane;
    double t = (r < pw && w < pw && w <= r) ? A[(size_t)(k0 + r) * d + k0 + w] : 0.0;
    panel_sync_init(ps);
    __syncthreads();
    if (w >= pw) return;
    for (int jj = 0; jj < w; ++jj) {
        if (!wait_col(&ps.bar[jj], 0u, &ps.abort_flag, J.status)) break;
        t = __fma_rn(-ps.Zs[jj][lane], ps.Zs[jj][w], t);
    }
    // pivot on lane w, division below it
    double piv = 0.0, rpiv = 0.0;
    if (lane == w) {
        if (!(t > tol_abs)) atomicOr(J.status, kStatusPivot);
        const double a = t > 0.0 ? t : 1.0;
        if (J.tc) {
            // tensor-core mode: y ~ 1/sqrt(a) within about half an ulp; L_ww = a y and L_rw = t_rw y
            // (each within about an ulp of the correctly rounded square root and quotient) come
            // from one multiplication on every lane, a shorter chain than a square root
            // followed by a division
            rpiv = rsqrt_near(a);
            t = a;
        } else {
            piv = __dsqrt_rn(a);
        }
    }
    if (J.tc) {
        rpiv = __shfl_sync(0xffffffffu, rpiv, w);
        if (lane >= w && lane < pw) t = __dmul_rn(t, rpiv);
    } else {
        piv = __shfl_sync(0xffffffffu, piv, w);
        if (lane == w) t = piv;
        else if (lane > w && lane < pw) t = __ddiv_rn(t, piv);
    }
    publish(ps, w, lane, (lane >= w && lane < pw) ? t : 0.0);
    if (r < pw && w <= r) A[(size_t)(k0 + r) * d + k0 + w] = t;
}

// Rows below the diagonal block of panel p, 32 per block: L_r,jj = (A_r,jj - sum_{k<jj}
// L_r,k L_jj,k) / L_jj,jj over the panel's columns, against the finished diagonal block.
__global__ void __launch_bounds__(kP * kPW) k_chol_below(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    double* __restrict__ A = J.Lm;
    __shared__ double Lc[kP][kP + 1];  // Lc[jj][kk] = L_{k0+kk, k0+jj}, kk >= jj
    __shared__ double Ld[kP], Yd[kP];
    __shared__ PanelSync ps;
    {
        const int kk = threadIdx.x / kP, jj = threadIdx.x % kP;  // lanes along a row of L: contiguous loads
        Lc[jj][kk] = (kk < pw && kk >= jj) ? A[(size_t)(k0 + kk) * d + k0 + jj] : 0.0;
    }
    if (threadIdx.x < pw) {
        const double l = A[(size_t)(k0 + threadIdx.x) * d + k0 + threadIdx.x];
        Ld[threadIdx.x] = l;
        Yd[threadIdx.x] = __ddiv_rn(1.0, l);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = k0 + pw + (int)lb * 32 + lane;
    const double t0 = (r < d && w < pw) ? A[(size_t)r * d + k0 + w] : 0.0;
    panel_sync_init(ps);
    __syncthreads();
    const double t = eliminate_panel_rows(t0, pw, w, lane, Lc, Ld, Yd, ps, r < d, J.status, J.tc != 0);
    if (r < d && w < pw) A[(size_t)r * d + k0 + w] = t;
}

// Look-ahead part of the trailing update after panel p: the diagonal block of panel p + 1
// (rows and columns [k0 + pw, k0 + pw + pw1)) receives A_ij -= L_ik L_jk for k in panel p
// (ascending), the operations of k_chol_trailing's tile (0, 0), so that the next diagonal
// block can be factored while the rest of the trailing update runs. One block (one warp) per
// row i of the tile, lane = column j <= i.
__global__ void __launch_bounds__(32) k_chol_lookahead(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    const int r0 = k0 + pw;
    double* __restrict__ A = J.Lm;
    const int i = r0 + (int)lb, j = r0 + (int)threadIdx.x;
    // rows r0 .. i of panel p through shared memory, each row read contiguously (lane = k; a
    // lane per row would touch 32 rows d apart in every load)
    __shared__ double tile[kP][kP + 1];
    {
        double v[kP];  // all row loads in flight before the first store
#pragma unroll
        for (int q = 0; q < kP; ++q)
            v[q] = (q <= i - r0 && (int)threadIdx.x < pw) ? A[(size_t)(r0 + q) * d + k0 + threadIdx.x] : 0.0;
#pragma unroll
        for (int q = 0; q < kP; ++q) tile[q][threadIdx.x] = v[q];
    }
    __syncwarp();
    if (j > i) return;
    // every operand is loaded before the chain of dependent FMAs starts
    double li[kP], lj[kP];
#pragma unroll
    for (int kk = 0; kk < kP; ++kk) {
        li[kk] = tile[i - r0][kk];
        lj[kk] = tile[j - r0][kk];
    }
    double v = A[(size_t)i * d + j];
#pragma unroll
    for (int kk = 0; kk < kP; ++kk)
        if (kk < pw) v = __fma_rn(-li[kk], lj[kk], v);
    A[(size_t)i * d + j] = v;
}

// Trailing update after panel p: A_ij -= L_ik L_jk for k in the panel (ascending), for
// k0 + pw <= j <= i < d. 32 x 32 tiles, lower-triangle tiles only: tile (ti, tj) has index
// b = ti (ti + 1) / 2 + tj, tj <= ti, and local block lb covers tile b = lb + 1 (tile 0, the
// next panel's diagonal block, is k_chol_lookahead's).
__global__ void __launch_bounds__(256) k_chol_trailing(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    double* __restrict__ A = J.Lm;
    const unsigned b = lb + 1;
    int ti = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= (int)b) ++ti;
    while (ti * (ti + 1) / 2 > (int)b) --ti;
    const int tj = (int)b - ti * (ti + 1) / 2;
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
        for (int kk = 0; kk < pw; ++kk) v = __fma_rn(-Li[ii][kk], Lj[jj][kk], v);
        A[(size_t)i * d + j] = v;
    }
}

// Panel p of the forward substitution Zc = Xc L^{-T}, in place in ZT (n x d row-major:
// working values, final Zc on exit): 32 rows per block, eliminated against the panel's
// diagonal block of L (z_ij = (t_ij - sum_{k<j} L_jk z_ik) / L_jj, subtractions in ascending k).
__global__ void __launch_bounds__(kP * kPW) k_fwd_panel(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    const double* __restrict__ L = J.Lm;
    double* __restrict__ T = J.ZT;
    __shared__ double Lc[kP][kP + 1];  // Lc[jj][kk] = L_{k0+kk, k0+jj}, kk >= jj
    __shared__ double Ld[kP], Yd[kP];
    __shared__ PanelSync ps;
    {
        const int kk = threadIdx.x / kP, jj = threadIdx.x % kP;  // lanes along a row of L: contiguous loads
        Lc[jj][kk] = (kk < pw && kk >= jj) ? L[(size_t)(k0 + kk) * d + k0 + jj] : 0.0;
    }
    if (threadIdx.x < pw) {
        const double l = L[(size_t)(k0 + threadIdx.x) * d + k0 + threadIdx.x];
        Ld[threadIdx.x] = l;
        Yd[threadIdx.x] = __ddiv_rn(1.0, l);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = (int)lb * 32 + lane;
    const double t0 = (i < n && w < pw) ? T[(size_t)i * d + k0 + w] : 0.0;
    panel_sync_init(ps);
    __syncthreads();
    const double t = eliminate_panel_rows(t0, pw, w, lane, Lc, Ld, Yd, ps, i < n, J.status, J.tc != 0);
    if (i < n && w < pw) T[(size_t)i * d + k0 + w] = t;
}

// T_ij -= L_jk z_ik for k in panel p (ascending), j >= k0 + pw. 32 x 32 tiles, local block
// b = (row tile) * (column tiles) + (column tile).
// Columns a panel's trailing update reaches: all later ones, or in tensor-core mode those of
// its own kFwdBlock-column block (later blocks receive the block's contributions at once, from
// digit products, after its last panel).
__host__ __device__ inline int fwd_trailing_end(const PrepJob& j, int k0)
{
    if (!j.tc) return j.d;
    const int e = (k0 / kFwdBlock + 1) * kFwdBlock;
    return e < j.d ? e : j.d;
}

__global__ void __launch_bounds__(256) k_fwd_trailing(PJ_ARGS, int p)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d, k0 = kP * p;
    const int pw = (d - k0) < kP ? (d - k0) : kP;
    const double* __restrict__ L = J.Lm;
    double* __restrict__ T = J.ZT;
    const int cend = fwd_trailing_end(J, k0);
    const unsigned gx = (unsigned)((cend - k0 - pw + 31) / 32);
    __shared__ double Zi[32][kP + 1], Lj[32][kP + 1];
    const int i0 = 32 * (int)(lb / gx), j0 = k0 + pw + 32 * (int)(lb % gx);
    for (int e = threadIdx.x; e < 32 * kP; e += blockDim.x) {
        const int rr = e / kP, kk = e % kP;
        Zi[rr][kk] = (i0 + rr < n && kk < pw) ? T[(size_t)(i0 + rr) * d + k0 + kk] : 0.0;
        Lj[rr][kk] = (j0 + rr < cend && kk < pw) ? L[(size_t)(j0 + rr) * d + k0 + kk] : 0.0;
    }
    __syncthreads();
    const int jj = threadIdx.x & 31;
    for (int ii = threadIdx.x >> 5; ii < 32; ii += blockDim.x >> 5) {
        const int i = i0 + ii, j = j0 + jj;
        if (i >= n || j >= cend) continue;
        double v = T[(size_t)i * d + j];
        for (int kk = 0; kk < pw; ++kk) v = __fma_rn(-Lj[jj][kk], Zi[ii][kk], v);
        T[(size_t)i * d + j] = v;
    }
}

__global__ void k_copy_zc(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const size_t idx = (size_t)lb * blockDim.x + threadIdx.x;
    if (idx < (size_t)J.n * J.d) J.Zc64[idx] = J.ZT[idx];
}

// qexp_j such that |Zc_ij * 2^qexp_j| <= 2^kQBits for every i. Block (32, kRG): 32 columns,
// the rows split over kRG thread rows (a maximum does not depend on the order of its operands).
constexpr int kRG = 16;

__global__ void __launch_bounds__(32 * kRG) k_qexp(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d;
    const int j = (int)lb * 32 + threadIdx.x;
    __shared__ unsigned long long part[kRG][32];
    // max |Zc_ij| as an integer maximum of the magnitudes' bit patterns (no FP64 compares)
    unsigned long long mb = 0ull;
    if (j < d) {
        const unsigned long long* z = reinterpret_cast<const unsigned long long*>(J.Zc64) + j;
#pragma unroll 8
        for (int i = threadIdx.y; i < n; i += kRG) {
            const unsigned long long b = z[(size_t)i * d] & 0x7FFFFFFFFFFFFFFFull;
            mb = b > mb ? b : mb;
        }
    }
    part[threadIdx.y][threadIdx.x] = mb;
    __syncthreads();
    if (threadIdx.y != 0 || j >= d) return;
    for (int g = 1; g < kRG; ++g) mb = part[g][threadIdx.x] > mb ? part[g][threadIdx.x] : mb;
    const double mx = __longlong_as_double((long long)mb);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e with f in [0.5, 1): mx < 2^e
    J.qexp[j] = (mx > 0.0) ? (kQBits - e) : 0;
}

// K-order derived arrays (p = K position, u = unit at p); every element of Z32, Zhi, Zlo and
// Q is written (zero at padding positions).
__global__ void k_derive(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d, kpad = J.kpad, dpad32 = J.dpad32;
    const size_t idx = (size_t)lb * blockDim.x + threadIdx.x;
    if (idx >= (size_t)kpad * dpad32) return;
    const int p = (int)(idx / dpad32), j = (int)(idx % dpad32);
    const int u = unit_of_kpos(p);
    const double z = (u < n && j < d) ? J.Zc64[(size_t)u * d + j] : 0.0;
    J.Z32[idx] = (float)z;
    if (j < d) {
        const __nv_bfloat16 hi = __double2bfloat16(z);
        const __nv_bfloat16 lo = __double2bfloat16(z - (double)__bfloat162float(hi));
        J.Zhi[(size_t)j * kpad + p] = hi;
        J.Zlo[(size_t)j * kpad + p] = lo;
        J.Q[(size_t)p * d + j] = llrint(ldexp(z, J.qexp[j]));
    }
}

// Balanced base-4096 digits of Q: Q = sum_{k<4} q_k 4096^k with q_k in [-2048, 2047], plane
// k stored K-major as FP16 (integers of this size are exact): Zq[(k d + j) kpad + p].
__global__ void k_digits(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, kpad = J.kpad;
    const size_t idx = (size_t)lb * blockDim.x + threadIdx.x;
    if (idx >= (size_t)kpad * d) return;
    const int j = (int)(idx / kpad), p = (int)(idx % kpad);
    long long v = J.Q[(size_t)p * d + j];
    constexpr int base = 1 << kDigitBits, half = base / 2;
    for (int k = 0; k < kDigitPlanes; ++k) {
        int q = (int)(v & (base - 1));
        if (q >= half) q -= base;
        v = (v - q) >> kDigitBits;
        J.Zq[((size_t)k * d + j) * kpad + p] = __float2half_rn((float)q);
    }
}

// Qsum_j = sum_p Q_pj: integer additions, exact in any order, so the K positions are split
// over kRG thread rows as in k_qexp.
__global__ void __launch_bounds__(32 * kRG) k_qsum(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int d = J.d, kpad = J.kpad;
    const int j = (int)lb * 32 + threadIdx.x;
    __shared__ long long part[kRG][32];
    long long s = 0;
    if (j < d) {
#pragma unroll 8
        for (int p = threadIdx.y; p < kpad; p += kRG) s += J.Q[(size_t)p * d + j];
    }
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y != 0 || j >= d) return;
    for (int g = 1; g < kRG; ++g) s += part[g][threadIdx.x];
    J.Qsum[j] = s;
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
// One block per column; eps[j] and eps[d + j] receive the two paths' terms.
__global__ void __launch_bounds__(256) k_band_cols(PJ_ARGS)
{
    unsigned lb;
    const PrepJob& J = job_of(jobs, prefix, E, lb);
    const int n = J.n, d = J.d, kused = J.kused;
    const double* __restrict__ Z = J.Zc64;
    // thread t covers K positions [t * per, (t + 1) * per)
    __shared__ double ws1[8], ws2[8], wacc[8], wr32[8], wrtc[8];
    const int j = (int)lb;
    const int per = (kused + 255) / 256;
    const int p0 = threadIdx.x * per;
    const double pi = (double)J.n1 / n;
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
        // the standard-deviation term in FP32 rounded upward (never below the FP64 value beyond
        // that product's own rounding; FP32 square roots cost no FP64 instructions)
        acc += fabs(pi * s1) + kBandLambda * (double)__fsqrt_ru(__double2float_ru(vf * s2)) + fabs(z);
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
        J.eps[j] = R32 + ldexp(A, -24);
        J.eps[d + j] = RTC + 2.0 * ldexp(A, -23);
    }
}

BandConsts band_from_eps(const double* eps, double c_M, int64_t d)
{
    double ss = 0.0;
    for (int64_t j = 0; j < d; ++j) ss += eps[j] * eps[j];
    const double en = sqrt(ss);
    const double u = ldexp(1.0, -24);
    const double g = (double)(d + 2) * u / (1.0 - (double)(d + 2) * u);
    BandConsts b;
    b.lin = 2.0 * sqrt(c_M) * en;
    b.quad = 3.0 * c_M * ss;
    b.rel = g;
    return b;
}

// C(c, m) for c, m < 64 at [c * 64 + m] (Pascal's rule; every entry fits in 64 bits), built once
const uint64_t* binom_table()
{
    static const std::vector<uint64_t> tab = [] {
        std::vector<uint64_t> t(64 * 64, 0);
        for (int c = 0; c < 64; ++c) {
            t[(size_t)c * 64] = 1;
            for (int m = 1; m <= c; ++m)
                t[(size_t)c * 64 + m] = t[(size_t)(c - 1) * 64 + m - 1] + t[(size_t)(c - 1) * 64 + m];
        }
        return t;
    }();
    return tab.data();
}

// Block counts of the launches of one job (0: the job has no work in that launch).
struct JobBlocks {
    static unsigned colmean(const PrepJob& j) { return (unsigned)ceil_div(j.d, 32); }
    static unsigned cols32(const PrepJob& j) { return (unsigned)ceil_div(j.d, 32); }
    static unsigned center(const PrepJob& j) { return (unsigned)(((size_t)j.n * j.d + 255) / 256); }
    static unsigned cov(const PrepJob& j) { return j.tc ? 0u : (unsigned)(ceil_div(j.d, 32) * ceil_div(j.d, 8)); }
    static unsigned cov_exp(const PrepJob& j) { return j.tc ? cov_tc_exp_blocks(j.n, j.d) : 0u; }
    static unsigned cov_digits(const PrepJob& j) { return j.tc ? cov_tc_digit_blocks(j.n, j.d) : 0u; }
    static unsigned cov_units(const PrepJob& j) { return j.tc ? cov_tc_units(j.n, j.d) : 0u; }
    static unsigned cov_finish(const PrepJob& j) { return j.tc ? cov_tc_finish_blocks(j.n, j.d) : 0u; }
    static unsigned one(const PrepJob&) { return 1u; }
    static unsigned init_L(const PrepJob& j) { return (unsigned)(((size_t)j.d * j.d + 255) / 256); }
    static unsigned chol_diag(const PrepJob& j, int p)
    {
        return (j.whiten == FRR_DIAG || kP * p >= j.d) ? 0u : 1u;
    }
    static unsigned chol_below(const PrepJob& j, int p)
    {
        const int k0 = kP * p;
        if (j.whiten == FRR_DIAG || k0 >= j.d) return 0u;
        const int pw = std::min(kP, j.d - k0), below = j.d - k0 - pw;
        return below > 0 ? (unsigned)ceil_div(below, 32) : 0u;
    }
    static unsigned chol_lookahead(const PrepJob& j, int p)
    {
        const int k0 = kP * p;
        if (j.whiten == FRR_DIAG || k0 >= j.d) return 0u;
        const int pw = std::min(kP, j.d - k0), below = j.d - k0 - pw;
        return (unsigned)std::max(0, std::min(kP, below));
    }
    static unsigned chol_trailing(const PrepJob& j, int p)
    {
        const int k0 = kP * p;
        if (j.whiten == FRR_DIAG || k0 >= j.d) return 0u;
        const int pw = std::min(kP, j.d - k0), below = j.d - k0 - pw;
        const unsigned t = below > 0 ? (unsigned)ceil_div(below, 32) : 0u;
        return t > 0 ? t * (t + 1) / 2 - 1 : 0u;  // every tile but the look-ahead one
    }
    static unsigned fwd_panel(const PrepJob& j, int p) { return kP * p < j.d ? (unsigned)ceil_div(j.n, 32) : 0u; }
    static unsigned fwd_trailing(const PrepJob& j, int p)
    {
        const int k0 = kP * p;
        if (k0 >= j.d) return 0u;
        const int pw = std::min(kP, j.d - k0), below = fwd_trailing_end(j, k0) - k0 - pw;
        return below > 0 ? (unsigned)(ceil_div(below, 32) * ceil_div(j.n, 32)) : 0u;
    }
    // the tensor-core update after the last panel of each kFwdBlock-column block (tensor-core mode)
    static unsigned fwd_xdigits(const PrepJob& j, int p) { return (j.tc && p % (kFwdBlock / kP) == kFwdBlock / kP - 1) ? fwd_tc_digit_blocks(j.n, j.d, p / (kFwdBlock / kP)) : 0u; }
    static unsigned fwd_xunits(const PrepJob& j, int p) { return (j.tc && p % (kFwdBlock / kP) == kFwdBlock / kP - 1) ? fwd_tc_units(j.n, j.d, p / (kFwdBlock / kP)) : 0u; }
    static unsigned fwd_xapply(const PrepJob& j, int p) { return (j.tc && p % (kFwdBlock / kP) == kFwdBlock / kP - 1) ? fwd_tc_apply_blocks(j.n, j.d, p / (kFwdBlock / kP)) : 0u; }
    static unsigned derive(const PrepJob& j) { return (unsigned)(((size_t)j.kpad * j.dpad32 + 255) / 256); }
    static unsigned digits(const PrepJob& j) { return (unsigned)(((size_t)j.kpad * j.d + 255) / 256); }
    static unsigned band(const PrepJob& j) { return (unsigned)j.d; }
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// ---- launch sequences kept as CUDA graphs ----------------------------------------------
// One experiment's preparation is ~200 dependent launches on three streams, tied together by
// events. Replayed from a graph they follow each other sooner on the device than when the
// launches and event records are enqueued one by one (frr_init 2.20 -> 1.99 ms, medians, at
// n = d = 1000), and the host enqueues one graph instead of ~200 launches (~0.8 ms). The
// sequence depends only on the shape and the options, and every kernel finds its arrays
// through the device job table, so the first call of a shape captures it into a graph that
// keeps its own temporary block, and later calls of that shape replay it (the covariate
// upload, the job tables and the read-back stay outside the graph). Single experiments
// only: a batch's launches cover all of its experiments, and its block can be gigabytes. At
// most kMaxPrepGraphs shapes per device are kept (least recently used first out).
struct PrepGraph {
    int key[8];
    int device;
    void* owner;           // CUDA context the block and the graph were made in
    char* base;            // the temporary block (prep_run_batch's layout for this shape)
    size_t bytes;
    cudaGraphExec_t exec;  // null until the first call of the shape has been captured
    bool busy, broken;
    unsigned long long last_use;
};
constexpr int kMaxPrepGraphs = 4;
constexpr size_t kMaxPrepGraphBytes = (size_t)512 << 20;
std::mutex g_graph_mutex;
std::vector<PrepGraph*> g_graphs;
unsigned long long g_graph_tick = 0;

// The entry of this shape, reserved for the caller until prep_graph_release, or null: its
// entry is in use by another thread or failed before, the block would be too large, or it
// cannot be allocated (the caller then takes a block from the pool and enqueues the launches
// itself). `device` is the current device.
PrepGraph* prep_graph_acquire(const PrepJob& J, int device, size_t bytes)
{
    if (bytes > kMaxPrepGraphBytes) return nullptr;
    void* owner = current_cuda_context();
    if (!owner) return nullptr;
    const int key[8] = {J.n, J.d, J.n1, J.whiten, J.kpad, J.dpad32, J.kused, J.tc};
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    // entries made in a context that no longer exists (cudaDeviceReset): their memory and graph
    // went with it, so they are forgotten, not freed
    for (size_t i = 0; i < g_graphs.size();) {
        PrepGraph* g = g_graphs[i];
        if (g->device == device && g->owner != owner && !g->busy) {
            delete g;
            g_graphs.erase(g_graphs.begin() + (long)i);
        } else {
            ++i;
        }
    }
    int on_device = 0;
    for (PrepGraph* g : g_graphs) {
        if (g->device != device) continue;
        ++on_device;
        if (std::equal(key, key + 8, g->key)) {
            if (g->busy || g->broken || g->bytes != bytes) return nullptr;
            g->busy = true;
            g->last_use = ++g_graph_tick;
            return g;
        }
    }
    if (on_device >= kMaxPrepGraphs) {
        PrepGraph* lru = nullptr;
        for (PrepGraph* g : g_graphs)
            if (g->device == device && !g->busy && (!lru || g->last_use < lru->last_use)) lru = g;
        if (!lru) return nullptr;
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        cudaFree(lru->base);  // idle: its last call synchronised before releasing it
        cudaGetLastError();
        g_graphs.erase(std::find(g_graphs.begin(), g_graphs.end(), lru));
        delete lru;
    }
    char* base = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&base), bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    PrepGraph* g = new PrepGraph{};
    std::copy(key, key + 8, g->key);
    g->device = device;
    g->owner = owner;
    g->base = base;
    g->bytes = bytes;
    g->busy = true;
    g->last_use = ++g_graph_tick;
    g_graphs.push_back(g);
    return g;
}

// Ends the caller's use of an entry (after its stream has been synchronised). An entry whose
// call failed is not used again.
void prep_graph_release(PrepGraph* g, bool ok)
{
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    if (!ok) g->broken = true;
    g->busy = false;
}

}  // namespace

frr_status prep_run_batch(frr_ctx* const* ctxs, const double* const* X_host, int E, cudaStream_t s,
                          cudaStream_t aux, frr_status* st_out)
{
    if (E < 1) return FRR_OK;
    const int device = ctxs[0]->device;
    cudaMemPool_t pool = temp_pool(device);
    if (pool == nullptr) return FRR_E_CUDA;

    // ---- one temporary allocation: per-job arrays, status words, job table, prefixes
    std::vector<PrepJob> jobs((size_t)E);
    std::vector<size_t> joff((size_t)E);
    size_t bytes = 0;
    int max_panels = 0;
    for (int e = 0; e < E; ++e) {
        const frr_ctx* c = ctxs[e];
        const size_t n = (size_t)c->n, d = (size_t)c->d;
        joff[(size_t)e] = bytes;
        bytes += 3 * align256(n * d * 8) + 2 * align256(d * d * 8) + 2 * align256(d * 8) + align256(4 * 8) +
                 align256(2 * d * 8);
        if (c->opts.prep == FRR_PREP_TENSOR) {
            // covariance: digit planes, exponents, int64 sums; forward substitution (d > kFwdBlock): the
            // two plane sets, row exponents, int64 sums
            bytes += align256(cov_tc_plane_bytes((int)n, (int)d)) + align256(d * 4) + align256(d * d * 8);
            if (d > (size_t)kFwdBlock)
                bytes += align256(fwd_tc_plane_bytes_a((int)n)) + align256(fwd_tc_plane_bytes_b((int)d)) +
                         align256(n * 4) + align256(d * 4) + align256(n * d * 8);
        }
        max_panels = std::max(max_panels, ceil_div(c->d, kP));
    }
    // the covariance jobs and their tensor maps (64-byte aligned)
    const size_t covjob_off = bytes;
    bytes += align256((size_t)E * sizeof(CovJob));
    const size_t fwdjob_off = bytes;
    bytes += align256((size_t)E * sizeof(FwdJob));
    const size_t maps_off = bytes;  // per job: the covariance's map, then the forward substitution's two
    bytes += align256((size_t)E * 3 * sizeof(CUtensorMap));
    const size_t status_off = bytes;
    bytes += align256((size_t)E * sizeof(int));
    const size_t table_off = bytes;
    bytes += align256((size_t)E * sizeof(PrepJob));
    // prefix arrays of every launch, in launch order
    std::vector<unsigned> pref;
    std::vector<size_t> pref_at;
    auto add_launch = [&](auto count) {
        pref_at.push_back(pref.size());
        unsigned acc = 0;
        for (int e = 0; e < E; ++e) {
            pref.push_back(acc);
            acc += count(jobs[(size_t)e]);
        }
        pref.push_back(acc);
    };
    char* base = nullptr;
    {
        // fill the job table (pointers relative to the future base; fixed up below)
        for (int e = 0; e < E; ++e) {
            const frr_ctx* c = ctxs[e];
            PrepJob& J = jobs[(size_t)e];
            J.n = (int)c->n; J.d = (int)c->d; J.n1 = (int)c->n1; J.whiten = c->opts.whiten;
            J.kpad = c->kpad; J.dpad32 = c->dpad32; J.kused = c->kused; J.ridge = c->opts.ridge;
            J.tc = c->opts.prep == FRR_PREP_TENSOR ? 1 : 0;
            J.Zc64 = c->Zc64; J.Z32 = c->Z32; J.Zhi = c->Zhi; J.Zlo = c->Zlo; J.Zq = c->Zq;
            J.Q = c->Q; J.Qsum = c->Qsum; J.qexp = c->qexp;
        }
    }
    add_launch(JobBlocks::colmean);
    add_launch(JobBlocks::center);
    add_launch(JobBlocks::cov);
    add_launch(JobBlocks::cov_exp);
    add_launch(JobBlocks::cov_digits);
    add_launch(JobBlocks::cov_units);
    add_launch(JobBlocks::cov_finish);
    add_launch(JobBlocks::one);
    add_launch(JobBlocks::init_L);
    for (int p = 0; p < max_panels; ++p) {
        add_launch([p](const PrepJob& j) { return JobBlocks::chol_diag(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::chol_below(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::fwd_panel(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::chol_trailing(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::fwd_trailing(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::chol_lookahead(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::fwd_xdigits(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::fwd_xunits(j, p); });
        add_launch([p](const PrepJob& j) { return JobBlocks::fwd_xapply(j, p); });
    }
    add_launch(JobBlocks::center);  // Zc copy
    add_launch(JobBlocks::cols32);  // qexp
    add_launch(JobBlocks::derive);
    add_launch(JobBlocks::cols32);  // qsum
    add_launch(JobBlocks::digits);
    add_launch(JobBlocks::band);
    const size_t pref_off = bytes;
    bytes += align256(pref.size() * sizeof(unsigned));

    PrepGraph* graph = (E == 1) ? prep_graph_acquire(jobs[0], device, bytes) : nullptr;
    bool capturing = false;  // the launches are being captured into graph
    frr_status rc = FRR_OK;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t up[2] = {nullptr, nullptr};  // the covariate upload on the second stream
    cudaStream_t ts = nullptr;  // the Cholesky's trailing updates
    std::vector<int> h_status((size_t)E, 0);
    std::vector<std::vector<double>> h_eps((size_t)E);
    std::vector<CovJob> cjobs((size_t)E);
    std::vector<FwdJob> fjobs((size_t)E);
    std::vector<CUtensorMap> cmaps((size_t)E * 3);
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        rc = (e == cudaErrorMemoryAllocation) ? FRR_E_NOMEM : FRR_E_CUDA;
    };
#define PREP_CHECK(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { fail(_e); goto cleanup; } } while (0)
    if (graph)
        base = graph->base;
    else
        PREP_CHECK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&base), bytes, pool, s));
    for (int e = 0; e < E; ++e) {
        PrepJob& J = jobs[(size_t)e];
        const size_t n = (size_t)J.n, d = (size_t)J.d;
        char* q = base + joff[(size_t)e];
        auto take = [&](size_t b) { char* r = q; q += align256(b); return reinterpret_cast<double*>(r); };
        J.X = take(n * d * 8); J.Xc = take(n * d * 8); J.ZT = take(n * d * 8);
        J.S = take(d * d * 8); J.Lm = take(d * d * 8);
        J.xbar = take(d * 8); J.Adiag = take(d * 8); J.scal = take(4 * 8); J.eps = take(2 * d * 8);
        J.status = reinterpret_cast<int*>(base + status_off) + e;
        h_eps[(size_t)e].resize(2 * d);
        CovJob& C = cjobs[(size_t)e];
        C = CovJob{};
        if (J.tc) {
            C.n = J.n; C.d = J.d; C.npad = cov_tc_npad(J.n); C.dpad = cov_tc_dpad(J.d);
            C.Xc = J.Xc; C.S = J.S; C.status = J.status; C.rinv = 1.0 / (double)(J.n - 1);
            C.G = reinterpret_cast<__nv_bfloat16*>(take(cov_tc_plane_bytes(J.n, J.d)));
            C.cexp = reinterpret_cast<int*>(take(d * 4));
            C.acc = reinterpret_cast<long long*>(take(d * d * 8));
            C.gmap = reinterpret_cast<const CUtensorMap*>(base + maps_off) + 3 * e;
            if (!cov_tc_map(&cmaps[3 * (size_t)e], C.G, J.n, J.d)) { rc = FRR_E_CUDA; goto cleanup; }
        }
        FwdJob& F = fjobs[(size_t)e];
        F = FwdJob{};
        J.facc = nullptr;
        if (J.tc && J.d > kFwdBlock) {
            F.n = J.n; F.d = J.d; F.npadA = fwd_tc_npadA(J.n); F.dpadB = fwd_tc_dpadB(J.d);
            F.ZT = J.ZT; F.L = J.Lm; F.status = J.status;
            F.GA = reinterpret_cast<__nv_bfloat16*>(take(fwd_tc_plane_bytes_a(J.n)));
            F.GB = reinterpret_cast<__nv_bfloat16*>(take(fwd_tc_plane_bytes_b(J.d)));
            F.expA = reinterpret_cast<int*>(take(n * 4));
            F.expB = reinterpret_cast<int*>(take(d * 4));
            F.acc = reinterpret_cast<long long*>(take(n * d * 8));
            J.facc = F.acc;
            F.mapA = reinterpret_cast<const CUtensorMap*>(base + maps_off) + 3 * e + 1;
            F.mapB = reinterpret_cast<const CUtensorMap*>(base + maps_off) + 3 * e + 2;
            if (!fwd_tc_maps(&cmaps[3 * (size_t)e + 1], &cmaps[3 * (size_t)e + 2], F)) { rc = FRR_E_CUDA; goto cleanup; }
        }
    }
    PREP_CHECK(cudaMemsetAsync(base + status_off, 0, (size_t)E * sizeof(int), s));
    {
        // The covariates go up on both streams, which then use two copy engines (8 MB took
        // ~450 us on one and ~245 us on two): one experiment in two halves, a batch's
        // experiments each to the stream with fewer bytes queued.
        for (auto& ev : up) PREP_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        PREP_CHECK(cudaEventRecord(up[0], s));  // the block is allocated
        PREP_CHECK(cudaStreamWaitEvent(aux, up[0], 0));
        size_t queued[2] = {0, 0};
        for (int e = 0; e < E; ++e) {
            const size_t bytes = (size_t)jobs[(size_t)e].n * jobs[(size_t)e].d * 8;
            char* dst = reinterpret_cast<char*>(jobs[(size_t)e].X);
            const char* src = reinterpret_cast<const char*>(X_host[e]);
            if (E == 1) {
                const size_t half = bytes / 16 * 8;
                PREP_CHECK(cudaMemcpyAsync(dst, src, half, cudaMemcpyHostToDevice, s));
                PREP_CHECK(cudaMemcpyAsync(dst + half, src + half, bytes - half, cudaMemcpyHostToDevice, aux));
            } else {
                const int w = queued[1] < queued[0] ? 1 : 0;
                PREP_CHECK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, w ? aux : s));
                queued[w] += bytes;
            }
        }
        PREP_CHECK(cudaEventRecord(up[1], aux));
        PREP_CHECK(cudaStreamWaitEvent(s, up[1], 0));
    }
    PREP_CHECK(cudaMemcpyAsync(base + table_off, jobs.data(), (size_t)E * sizeof(PrepJob), cudaMemcpyHostToDevice, s));
    PREP_CHECK(cudaMemcpyAsync(base + covjob_off, cjobs.data(), (size_t)E * sizeof(CovJob), cudaMemcpyHostToDevice, s));
    PREP_CHECK(cudaMemcpyAsync(base + fwdjob_off, fjobs.data(), (size_t)E * sizeof(FwdJob), cudaMemcpyHostToDevice, s));
    PREP_CHECK(cudaMemcpyAsync(base + maps_off, cmaps.data(), (size_t)E * 3 * sizeof(CUtensorMap),
                               cudaMemcpyHostToDevice, s));
    PREP_CHECK(cudaMemcpyAsync(base + pref_off, pref.data(), pref.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                               s));
    if (graph && graph->exec) {
        PREP_CHECK(cudaGraphLaunch(graph->exec, s));
    } else {
        evs.assign(3, nullptr);  // [0]: rows below panel p final; [1]: trailing rest p done; [2]: fork / join
        for (auto& ev : evs) PREP_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        PREP_CHECK(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
        if (graph) {
            PREP_CHECK(prep_tc_setup(device));
            PREP_CHECK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            capturing = true;
        }
        const PrepJob* dj = reinterpret_cast<const PrepJob*>(base + table_off);
        const unsigned* dp = reinterpret_cast<const unsigned*>(base + pref_off);
        size_t li = 0;
        // blocks of launch li, and its prefix array on the device
        auto total = [&](size_t l) { return pref[pref_at[l] + (size_t)E]; };
        auto P = [&](size_t l) { return dp + pref_at[l]; };
        if (unsigned g = total(li)) k_colmean<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_center<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_cov<<<g, dim3(32, 8), 0, s>>>(dj, P(li), E);
        ++li;
        {
            const unsigned* cp[4] = {P(li), P(li + 1), P(li + 2), P(li + 3)};
            const unsigned ct[4] = {total(li), total(li + 1), total(li + 2), total(li + 3)};
            PREP_CHECK(cov_tc_launch(reinterpret_cast<const CovJob*>(base + covjob_off), cp, ct, E, device,
                                     ctxs[0]->num_sms, s));
            li += 4;
        }
        if (unsigned g = total(li)) k_diag<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_init_L<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        PREP_CHECK(cudaGetLastError());
        // Both factorisations are chains of latency-bound panels. Step p of the forward
        // substitution needs only column panel p of L, which is final once Cholesky panel
        // p is done (later trailing updates touch columns to its right), so it runs on the
        // second stream, one panel behind: the two chains overlap. Within the Cholesky, the
        // next panel's diagonal block gets panel p's update first (k_chol_lookahead) so that
        // it can be factored while the rest of the trailing update runs on a third stream;
        // the rows below panel p + 1 wait for that rest.
        // Three events serve every dependency: each wait is enqueued right after its record,
        // and a wait already enqueued is not affected by a later record of the same event.
        PREP_CHECK(cudaEventRecord(evs[2], s));
        PREP_CHECK(cudaStreamWaitEvent(aux, evs[2], 0));
        PREP_CHECK(cudaStreamWaitEvent(ts, evs[2], 0));
        for (int p = 0; p < max_panels; ++p) {
            const size_t ld = li, lp = li + 1, lf = li + 2, lt = li + 3, lft = li + 4, la = li + 5, lx = li + 6;
            li += 9;
            if (unsigned g = total(ld)) k_chol_diag<<<g, kP * kPW, 0, s>>>(dj, P(ld), E, p);
            if (p > 0) PREP_CHECK(cudaStreamWaitEvent(s, evs[1], 0));  // trailing rest p - 1
            if (unsigned g = total(lp)) k_chol_below<<<g, kP * kPW, 0, s>>>(dj, P(lp), E, p);
            PREP_CHECK(cudaEventRecord(evs[0], s));
            PREP_CHECK(cudaStreamWaitEvent(aux, evs[0], 0));
            PREP_CHECK(cudaStreamWaitEvent(ts, evs[0], 0));
            if (unsigned g = total(lf)) k_fwd_panel<<<g, kP * kPW, 0, aux>>>(dj, P(lf), E, p);
            if (unsigned g = total(la)) k_chol_lookahead<<<g, 32, 0, s>>>(dj, P(la), E, p);
            if (unsigned g = total(lt)) k_chol_trailing<<<g, 256, 0, ts>>>(dj, P(lt), E, p);
            PREP_CHECK(cudaEventRecord(evs[1], ts));
            if (unsigned g = total(lft)) k_fwd_trailing<<<g, 256, 0, aux>>>(dj, P(lft), E, p);
            if (p % (kFwdBlock / kP) == kFwdBlock / kP - 1) {
                // after the last panel of a kFwdBlock-column block: the block's contributions to every
                // later column, from digit products on the tensor cores (tensor-core mode)
                const unsigned* xp[3] = {P(lx), P(lx + 1), P(lx + 2)};
                const unsigned xt[3] = {total(lx), total(lx + 1), total(lx + 2)};
                if (xt[0] || xt[1] || xt[2])
                    PREP_CHECK(fwd_tc_launch(reinterpret_cast<const FwdJob*>(base + fwdjob_off), xp, xt, E, p / (kFwdBlock / kP),
                                             device, ctxs[0]->num_sms, aux));
            }
        }
        PREP_CHECK(cudaEventRecord(evs[2], aux));
        PREP_CHECK(cudaStreamWaitEvent(s, evs[2], 0));
        PREP_CHECK(cudaEventRecord(evs[2], ts));
        PREP_CHECK(cudaStreamWaitEvent(s, evs[2], 0));
        if (unsigned g = total(li)) k_copy_zc<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        // The band terms read only Zc: they run on the second stream beside the chain that
        // derives the balance and recheck copies (exponents, copies, sums, digit planes).
        PREP_CHECK(cudaEventRecord(evs[0], s));
        PREP_CHECK(cudaStreamWaitEvent(aux, evs[0], 0));
        if (unsigned g = total(li + 4)) k_band_cols<<<g, 256, 0, aux>>>(dj, P(li + 4), E);
        PREP_CHECK(cudaEventRecord(evs[1], aux));
        if (unsigned g = total(li)) k_qexp<<<g, dim3(32, kRG), 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_derive<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_qsum<<<g, dim3(32, kRG), 0, s>>>(dj, P(li), E);
        ++li;
        if (unsigned g = total(li)) k_digits<<<g, 256, 0, s>>>(dj, P(li), E);
        ++li;
        ++li;  // (k_band_cols, above)
        PREP_CHECK(cudaStreamWaitEvent(s, evs[1], 0));
        PREP_CHECK(cudaGetLastError());
        if (capturing) {
            cudaGraph_t g = nullptr;
            capturing = false;
            PREP_CHECK(cudaStreamEndCapture(s, &g));
            cudaGraphExec_t ex = nullptr;  // kept by the entry only once instantiated
            const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            PREP_CHECK(e);
            graph->exec = ex;
            PREP_CHECK(cudaGraphLaunch(graph->exec, s));
        }
    }
    // binomial tables for exact enumeration (only shapes that allow it read them); the host
    // table is static, so the copies need no synchronisation
    for (int e = 0; e < E; ++e)
        if (ctxs[e]->n <= kExactMaxN)
            PREP_CHECK(cudaMemcpyAsync(ctxs[e]->binom, binom_table(), 64 * 64 * sizeof(uint64_t),
                                       cudaMemcpyHostToDevice, s));
    // the single synchronisation of the preparation: pivot status and band inputs
    PREP_CHECK(cudaMemcpyAsync(h_status.data(), base + status_off, (size_t)E * sizeof(int), cudaMemcpyDeviceToHost, s));
    for (int e = 0; e < E; ++e)
        PREP_CHECK(cudaMemcpyAsync(h_eps[(size_t)e].data(), jobs[(size_t)e].eps, h_eps[(size_t)e].size() * 8,
                                   cudaMemcpyDeviceToHost, s));
    PREP_CHECK(cudaStreamSynchronize(s));
    for (int e = 0; e < E; ++e) {
        frr_ctx* c = ctxs[e];
        if (h_status[(size_t)e] != 0) {
            const int hs = h_status[(size_t)e];
            st_out[e] = (hs & kStatusNonFinite) ? FRR_E_ARG : (hs & kStatusTimeout) ? FRR_E_TIMEOUT : FRR_E_DEGENERATE;
            continue;
        }
        c->band32 = band_from_eps(h_eps[(size_t)e].data(), c->c_M, c->d);
        c->band_tc = band_from_eps(h_eps[(size_t)e].data() + c->d, c->c_M, c->d);
        st_out[e] = FRR_OK;
    }

cleanup:
#undef PREP_CHECK
    if (capturing) {  // failed while capturing: end the capture and keep nothing of it
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    // after a failure, work may still be in flight on the other streams (synchronised before
    // the trailing-update stream is destroyed and before the temporaries are released)
    if (rc != FRR_OK) {
        cudaStreamSynchronize(aux);
        if (ts) cudaStreamSynchronize(ts);
        if (graph) cudaStreamSynchronize(s);
        cudaGetLastError();
    }
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : up)
        if (ev) cudaEventDestroy(ev);
    if (ts) cudaStreamDestroy(ts);
    // stream-ordered release: no device-wide synchronisation
    if (base && !graph) cudaFreeAsync(base, s);
    if (graph) prep_graph_release(graph, rc == FRR_OK);
    if (rc != FRR_OK)
        for (int e = 0; e < E; ++e) st_out[e] = rc;
    return rc;
}

frr_status prep_run(frr_ctx* ctx, const double* X_host)
{
    frr_status st = FRR_OK;
    const frr_status rc = prep_run_batch(&ctx, &X_host, 1, ctx->stream, ctx->aux, &st);
    if (rc != FRR_OK) {
        ctx->failed = true;
        return rc;
    }
    return st;
}

}  // namespace frr
