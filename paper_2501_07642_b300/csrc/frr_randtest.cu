// frr_randtest.cu -- randomization test conditional on acceptance and its inversion.
//
// Sec. 2.3 (randomization_test) and Sec. 4 ("Design-based inference"): the
// observed statistic is compared with its distribution over the accepted
// assignments only; p >= 1/K because the observed assignment is one of them.
// Reading: sharp null Y_i(1) = Y_i(0) + tau, two-sided difference in means.
// Under that null the adjusted outcome is Y - tau w_obs, and for accepted
// assignment k
//   t_k(tau) = DiM_{w_k}(Y - tau w_obs) = a_k - tau b_k,
//   a_k = DiM_{w_k}(Y),  b_k = DiM_{w_k}(w_obs) = c_k / n1 - (n1 - c_k) / n0,
// with c_k = |w_k AND w_obs|; for the observed assignment b = 1 exactly. So a_k
// and b_k are formed once per key and each grid point costs K comparisons.
// The interval is [min, max] of the grid points with p > alpha.
#include "frr_internal.cuh"
#include "frr_gen.cuh"

#include <cstring>
#include <vector>

namespace frr {
namespace {

// a_k and b_k, one warp per key: lane l sums the treated and control outcomes of units
// l, l + 32, ... and the warp adds the lane sums in a fixed tree. (A single thread summing
// n units in order is a chain of n dependent FP64 additions, about 64 cycles each on B300.
// The different summation order changes a_k only in its last bits, so a comparison
// |t_k| >= |t_obs| can differ from an in-order evaluation only at numerical near-ties,
// which the tests allow and the oracle flags.) b_k from popcounts.
__global__ void k_contrasts(const uint32_t* __restrict__ rows, int words, int64_t K, int64_t obs, int n, int n1,
                            const double* __restrict__ Y, double* __restrict__ a, double* __restrict__ b)
{
    pdl_wait();
    pdl_launch_dependents();
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= K) return;
    const uint32_t* row = rows + k * words;
    const uint32_t* orow = rows + obs * words;
    double s1 = 0.0, s0 = 0.0;
    for (int i = lane; i < n; i += 32) {
        const int p = kpos_of_unit(i);
        if ((row[p >> 5] >> (p & 31)) & 1u) s1 = __dadd_rn(s1, Y[i]);
        else s0 = __dadd_rn(s0, Y[i]);
    }
    int c = 0;
    for (int q = lane; q < words; q += 32) c += __popc(row[q] & orow[q]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        s1 = __dadd_rn(s1, __shfl_xor_sync(kFull, s1, off));
        s0 = __dadd_rn(s0, __shfl_xor_sync(kFull, s0, off));
        c += __shfl_xor_sync(kFull, c, off);
    }
    if (lane != 0) return;
    const int n0 = n - n1;
    a[k] = __dsub_rn(__ddiv_rn(s1, (double)n1), __ddiv_rn(s0, (double)n0));
    b[k] = __dsub_rn(__ddiv_rn((double)c, (double)n1), __ddiv_rn((double)(n1 - c), (double)n0));
}

// one CTA per grid point: count_g = #{k : |a_k - tau b_k| >= |a_obs - tau b_obs|}
__global__ void k_tau_grid(const double* __restrict__ a, const double* __restrict__ b, int64_t K, int64_t obs,
                           const double* __restrict__ tau, long long* __restrict__ count, double* __restrict__ p,
                           long long* __restrict__ near)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ long long sc[32], sn[32];
    const int g = blockIdx.x;
    const double t = tau[g];
    const double tobs = fabs(__dsub_rn(a[obs], __dmul_rn(t, b[obs])));
    long long cnt = 0, nr = 0;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const double tk = fabs(__dsub_rn(a[k], __dmul_rn(t, b[k])));
        cnt += (tk >= tobs) ? 1 : 0;
        nr += (fabs(tk - tobs) < 1e-12 * (tobs + 1.0)) ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        cnt += __shfl_xor_sync(kFull, cnt, off);
        nr += __shfl_xor_sync(kFull, nr, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sc[warp] = cnt; sn[warp] = nr; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long c = 0, m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { c += sc[w]; m += sn[w]; }
        count[g] = c;
        near[g] = m;
        p[g] = __ddiv_rn((double)c, (double)K);
    }
}

// [min, max] of the grid points with p > alpha; one warp (the FP64 comparisons of a single
// thread over T points form a long dependent chain on B300's narrow FP64 unit)
__global__ void k_interval(const double* __restrict__ p, const double* __restrict__ tau, int64_t T, double alpha,
                           double* __restrict__ out)
{
    pdl_wait();
    pdl_launch_dependents();
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t g = threadIdx.x; g < T; g += 32)
        if (p[g] > alpha) {
            lo = fmin(lo, tau[g]);
            hi = fmax(hi, tau[g]);
        }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(kFull, lo, off));
        hi = fmax(hi, __shfl_xor_sync(kFull, hi, off));
    }
    if (threadIdx.x == 0) {
        out[0] = (lo == INFINITY) ? NAN : lo;
        out[1] = (hi == -INFINITY) ? NAN : hi;
    }
}

}  // namespace

frr_status randtest_enqueue(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, bool keys_on_device, int64_t K,
                            int64_t obs, const double* Y, const double* tau, int64_t T, double alpha,
                            const double** dp_out, const long long** dcount_out, const double** dci_out)
{
    const bool exact = (seed == FRR_EXACT_SEED);
    const int n = (int)ctx->n;
    const int words = 4 * ctx->kb;
    // scratch: keys (K), rows (K x words), Y (n), tau (T), a (K), b (K), count (T), near (T), p (T), ci (2)
    const size_t bytes = (size_t)K * 8 + (size_t)K * words * 4 + 8 + (size_t)n * 8 + (size_t)T * 8 + (size_t)K * 16 +
                         (size_t)T * 24 + 16 + 64;
    FRR_TRY(ensure_device(ctx, &ctx->rt, &ctx->rt_bytes, bytes));
    char* base = static_cast<char*>(ctx->rt);
    uint64_t* dkeys = reinterpret_cast<uint64_t*>(base);
    double* dy = reinterpret_cast<double*>(dkeys + K);
    double* dtau = dy + n;
    double* da = dtau + T;
    double* db = da + K;
    double* dp = db + K;
    double* dci = dp + T;
    long long* dcount = reinterpret_cast<long long*>(dci + 2);
    long long* dnear = dcount + T;
    uint32_t* rows = reinterpret_cast<uint32_t*>(dnear + T);
    if (!keys_on_device)
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(dkeys, keys, (size_t)K * 8, cudaMemcpyHostToDevice, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(dy, Y, (size_t)n * 8, cudaMemcpyDefault, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(dtau, tau, (size_t)T * 8, cudaMemcpyDefault, ctx->stream));
    FRR_TRY(bits_launch(ctx, seed, exact, 0, (uint64_t)K, keys_on_device ? keys : dkeys, rows));
    FRR_CUDA_TRY(ctx, launch_pdl(k_contrasts, ceil_div(K, 4), 128, 0, ctx->stream, (const uint32_t*)rows, words, K, obs,
                                 n, (int)ctx->n1, (const double*)dy, da, db));
    FRR_CUDA_TRY(ctx, launch_pdl(k_tau_grid, (unsigned)T, 256, 0, ctx->stream, (const double*)da, (const double*)db, K,
                                 obs, (const double*)dtau, dcount, dp, dnear));
    FRR_CUDA_TRY(ctx, launch_pdl(k_interval, 1, 32, 0, ctx->stream, (const double*)dp, (const double*)dtau, T, alpha,
                                 dci));
    *dp_out = dp;
    *dcount_out = dcount;
    *dci_out = dci;
    return FRR_OK;
}

frr_status randtest_run(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, int64_t K, uint64_t obs_key,
                        const double* Y, const double* tau, int64_t T, double alpha, double* p_out,
                        int64_t* count_out, double* ci_lo, double* ci_hi)
{
    const bool exact = (seed == FRR_EXACT_SEED);
    const int n = (int)ctx->n;
    // host views of the inputs: host memory is read in place; device inputs are copied
    // back together (one synchronisation)
    const bool keys_dev = is_device_ptr(keys), y_dev = is_device_ptr(Y), tau_dev = is_device_ptr(tau);
    std::vector<uint64_t> hk_buf;
    std::vector<double> hy_buf, ht_buf;
    const uint64_t* hk = keys;
    const double* hy = Y;
    const double* ht = tau;
    if (keys_dev) {
        hk_buf.resize((size_t)K);
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk_buf.data(), keys, (size_t)K * 8, cudaMemcpyDeviceToHost, ctx->stream));
        hk = hk_buf.data();
    }
    if (y_dev) {
        hy_buf.resize((size_t)n);
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hy_buf.data(), Y, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        hy = hy_buf.data();
    }
    if (tau_dev) {
        ht_buf.resize((size_t)T);
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(ht_buf.data(), tau, (size_t)T * 8, cudaMemcpyDeviceToHost, ctx->stream));
        ht = ht_buf.data();
    }
    if (keys_dev || y_dev || tau_dev) FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t obs = -1;
    for (int64_t k = 0; k < K; ++k)
        if (hk[k] == obs_key) { obs = k; break; }
    if (obs < 0) return FRR_E_ARG;
    if (exact) {
        const uint64_t tot = binom_host((int)ctx->n, (int)ctx->n1);
        for (int64_t k = 0; k < K; ++k)
            if (hk[k] >= tot) return FRR_E_RANGE;
    }
    for (int i = 0; i < n; ++i) if (!isfinite(hy[i])) return FRR_E_ARG;
    for (int64_t g = 0; g < T; ++g) if (!isfinite(ht[g])) return FRR_E_ARG;

    // pinned staging of the host outputs: p (T), count (T), ci (2)
    FRR_TRY(ensure_host_pinned(ctx, (size_t)T * 16 + 16));
    const double* dp = nullptr;
    const long long* dcount = nullptr;
    const double* dci = nullptr;
    FRR_TRY(randtest_enqueue(ctx, seed, keys, keys_dev, K, obs, Y, tau, T, alpha, &dp, &dcount, &dci));
    // outputs: device ones copied on the stream, host ones through the pinned staging; one
    // synchronisation for all
    double* sp = static_cast<double*>(ctx->host_pinned);
    long long* scount = reinterpret_cast<long long*>(sp + T);
    double* sci = reinterpret_cast<double*>(scount + T);
    const bool p_dev = is_device_ptr(p_out);
    const bool c_dev = count_out != nullptr && is_device_ptr(count_out);
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(p_dev ? (void*)p_out : (void*)sp, dp, (size_t)T * 8,
                                      p_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (count_out)
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(c_dev ? (void*)count_out : (void*)scount, dcount, (size_t)T * 8,
                                          c_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(sci, dci, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (!p_dev) memcpy(p_out, sp, (size_t)T * 8);
    if (count_out && !c_dev) memcpy(count_out, scount, (size_t)T * 8);
    if (ci_lo) *ci_lo = sci[0];
    if (ci_hi) *ci_hi = sci[1];
    return FRR_OK;
}

}  // namespace frr
