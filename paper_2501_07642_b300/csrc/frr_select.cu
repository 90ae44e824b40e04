// frr_select.cu -- acceptance of the best q fraction (or of M <= a) with an exact
// answer, plus key replay helpers.
//
// Sec. 2.2 keeps the draws in the accepted q-quantile of M (or M <= a); the
// library breaks ties by the lower draw index. The bulk paths give an
// approximate M_hat with a per-draw error band |M_hat - M| <= band(M_hat).
// Selection therefore runs in two stages:
//   1. streaming filter: over the chunk's M_hat plus the retained set, bound
//      the K-th smallest M_hat from above by two grid-wide histogram levels on
//      its float bits (m_up >= M_(K)), form the cut T = U(m_up) with
//      U(m) = m + band(m), and keep every draw whose lower bound
//      L(m) = m - band(m) is <= T. Any draw among the true K best has
//      L <= M <= M_(K)(true) <= T, so the retained set always contains them.
//   2. exact-sum recheck of the retained draws (fixed-point Zc, exact integer
//      sums on the tensor cores, FP64 assembly), then the K smallest
//      (M64, draw index), reported in ascending draw order.
#include "frr_internal.cuh"
#include "frr_gen.cuh"

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <vector>

namespace frr {
namespace {

// ------------------------------------------------------------------ replay --
// One warp per draw, grid-stride; the count is read from count_dev when given (a count
// the host has not read back), else it is `count`.
template <int KB>
__global__ void k_bits(uint64_t seed, int exact, const uint64_t* __restrict__ binom, int n, int n1, uint64_t first,
                       uint64_t count, const long long* __restrict__ count_dev, const uint64_t* __restrict__ draws,
                       uint32_t* __restrict__ rows)
{
    pdl_wait();
    pdl_launch_dependents();
    // a device count can exceed the bound when the retained set overflowed its buffer (the
    // host then redoes the selection); only the entries within the bound exist
    const uint64_t cnt = count_dev ? std::min<uint64_t>((uint64_t)*count_dev, count) : count;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < cnt; w += nw) {
        const uint64_t draw = draws ? draws[w] : first + w;
        warp_draw_bits<KB>(exact != 0, seed, draw, n, n1, binom, rows + w * (4 * KB), lane);
    }
}

// Selection on caller-supplied unit words (word of unit i at words[i]); one warp.
template <int KB>
__global__ void k_words_select(const uint32_t* __restrict__ words, int n, int n1, uint32_t* __restrict__ row)
{
    const int lane = threadIdx.x & 31;
    uint32_t r[4 * KB];
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int u = 128 * k + 4 * lane + c;
            r[4 * k + c] = u < n ? words[u] : 0xffffffffu;
        }
    const SelectOutcome<KB> sel = warp_select_smallest<KB>(r, n, n1, lane);
    warp_store_bits<KB>(sel, r, row);
}

__global__ void k_unpack(const uint32_t* __restrict__ rows, int words, uint64_t count, int n, uint8_t* __restrict__ w)
{
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count * (uint64_t)n) return;
    const uint64_t b = idx / n;
    const int i = (int)(idx % n);
    const int p = kpos_of_unit(i);
    w[idx] = (uint8_t)((rows[b * words + (p >> 5)] >> (p & 31)) & 1u);
}

// ----------------------------------------------------------------- recheck --
// Exact treated sums S_T,j = sum_{i in T} Q_ij in int64 for G draws x 128 columns
// per CTA; S_C,j = S_all,j - S_T,j exactly, so an assignment and its complement
// swap (S_T, S_C). Per column: Delta_j = S_T 2^-q / n1 - S_C 2^-q / n0 (FP64) and the
// CTA writes the fixed-order partial sum of Delta_j^2 over its columns.
constexpr int RG = 8;     // draws per CTA
constexpr int RCOLS = 128;

template <int KB>
__global__ void __launch_bounds__(RCOLS)
k_recheck(const long long* __restrict__ Q, const long long* __restrict__ Qsum, const int* __restrict__ qexp, int d,
          int kused, int n, int n1, uint64_t seed, int exact, const uint64_t* __restrict__ binom,
          const uint64_t* __restrict__ draws, int64_t count, double* __restrict__ part, int ncb)
{
    constexpr int W = 4 * KB;
    __shared__ uint32_t rows[RG][W];
    __shared__ double red[RCOLS / 32][RG];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g0 = (int64_t)blockIdx.x * RG;
    for (int g = warp; g < RG; g += RCOLS / 32) {
        if (g0 + g < count) warp_draw_bits<KB>(exact != 0, seed, draws[g0 + g], n, n1, binom, rows[g], lane);
        else for (int q = lane; q < W; q += 32) rows[g][q] = 0u;
    }
    __syncthreads();
    const int j = blockIdx.y * RCOLS + threadIdx.x;
    double part_g[RG];
#pragma unroll
    for (int g = 0; g < RG; ++g) part_g[g] = 0.0;
    if (j < d) {
        long long acc[RG];
#pragma unroll
        for (int g = 0; g < RG; ++g) acc[g] = 0;
        for (int m = 0; m < kused / 32; ++m) {
            uint32_t bw[RG];
#pragma unroll
            for (int g = 0; g < RG; ++g) bw[g] = rows[g][m];
            const long long* qp = Q + (size_t)(32 * m) * d + j;
#pragma unroll 8
            for (int u = 0; u < 32; ++u) {
                const long long q = qp[(size_t)u * d];
#pragma unroll
                for (int g = 0; g < RG; ++g)
                    if ((bw[g] >> u) & 1u) acc[g] += q;
            }
        }
        const int e = qexp[j];
        const long long all = Qsum[j];
        const int n0 = n - n1;
#pragma unroll
        for (int g = 0; g < RG; ++g) {
            const double m1 = __ddiv_rn(ldexp((double)acc[g], -e), (double)n1);
            const double m0 = __ddiv_rn(ldexp((double)(all - acc[g]), -e), (double)n0);
            const double dl = __dsub_rn(m1, m0);
            part_g[g] = __dmul_rn(dl, dl);
        }
    }
    // fixed-order block reduction: warp butterfly, then warps in order
#pragma unroll
    for (int g = 0; g < RG; ++g) {
        double v = part_g[g];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, off));
        if (lane == 0) red[warp][g] = v;
    }
    __syncthreads();
    if (threadIdx.x < RG) {
        const int g = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < RCOLS / 32; ++w) v = __dadd_rn(v, red[w][g]);
        if (g0 + g < count) part[(g0 + g) * ncb + blockIdx.y] = v;
    }
}

// M64 = scale * (sum of the column-block partial sums, in block order) / denom
__global__ void k_recheck_sum(const double* __restrict__ part, int ncb, int64_t count,
                              const long long* __restrict__ count_dev, double scale, double denom,
                              double* __restrict__ M64)
{
    pdl_wait();
    pdl_launch_dependents();
    const int64_t cnt = count_dev ? (*count_dev < count ? *count_dev : count) : count;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cnt; c += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < ncb; ++b) s = __dadd_rn(s, part[c * ncb + b]);
        M64[c] = __ddiv_rn(__dmul_rn(scale, s), denom);
    }
}

// ---------------------------------------------------------- stream filter --
constexpr int SNT = 1024;

struct CutParams {
    double lin, quad, rel, safety;
};

__device__ __forceinline__ double lower_bound_m(const CutParams& cp, float v)
{
    const double m = (double)v;
    return m - band_value(cp.lin, cp.quad, cp.rel, cp.safety, m);
}

// largest non-negative float v with L(v) <= T, where L(v) = v - s (lin sqrt(v) + quad + rel v)
// is <= 0 near 0 and increasing after its minimum. With x = sqrt(v), L(v) = T is the
// quadratic (1 - s rel) x^2 - s lin x - (s quad + T) = 0; its root gives v, and the float
// result is stepped down until L(v) <= T holds and up while the next float still satisfies it.
__device__ float largest_v_below(const CutParams& cp, double T, uint32_t lo_bits)
{
    if (!(T < INFINITY)) return INFINITY;
    const double A = 1.0 - cp.safety * cp.rel, Bq = cp.safety * cp.lin, Cq = cp.safety * cp.quad + T;
    const double x = (Bq + sqrt(Bq * Bq + 4.0 * A * Cq)) / (2.0 * A);
    uint32_t v = __float_as_uint((float)(x * x));
    if (v < lo_bits) v = lo_bits;                 // L(lo) <= T holds by construction
    for (int i = 0; i < 64 && v > lo_bits && lower_bound_m(cp, __uint_as_float(v)) > T; ++i) --v;
    for (int i = 0; i < 64 && v < 0x7f7fffffu && lower_bound_m(cp, __uint_as_float(v + 1)) <= T; ++i) ++v;
    return __uint_as_float(v);
}

// Block-wide exclusive scan of one int per thread (SNT threads). Returns the
// exclusive prefix; *total gets the block sum.
__device__ int block_scan_excl(int v, int* ws, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = ws[lane];
        int si = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, si, off);
            if (lane >= off) si += y;
        }
        ws[lane] = si - s;
        if (lane == 31) ws[32] = si;
    }
    __syncthreads();
    const int res = ws[warp] + incl - v;
    *total = ws[32];
    __syncthreads();
    return res;
}

// ---- parallel selection of the cut over V = chunk (nc values) + retained (nr values)
// Two histogram levels on the float bit pattern (M_hat >= 0, so the bit order is the
// value order): bits [31:20] over all of V, then bits [19:8] inside the bin that holds
// the K-th smallest. The K-th smallest value lies below the upper edge m_up of the
// second-level bin, so T = U(m_up) >= U(M_(K)) is a safe cut; it is looser than the
// exact one by at most 2^-15 relative.
constexpr int kBins = 4096;
constexpr int kHistThreads = 256;

struct SelState {
    unsigned hist[2][kBins];
    unsigned prefix1, prefix2;
    long long krem;
    float cut;
    long long kept;
    // end-of-stream results, read back in one copy (see SelTail)
    long long nsel;
    double boundary[2];      // M64 of ranks K-1 and K (q mode)
    double max_rel, max_over_band, thr;
    int violations;
};

static_assert(offsetof(SelState, violations) - offsetof(SelState, nsel) == 48, "SelState tail layout");
static_assert(offsetof(SelState, nsel) - offsetof(SelState, kept) == sizeof(long long), "kept precedes the tail");

// the part of SelState read back by the host at the end of a stream
struct SelTail {
    long long nsel;
    double boundary[2];
    double max_rel, max_over_band, thr;
    int violations;
};
static_assert(offsetof(SelTail, violations) == 48, "SelTail layout");

__device__ __forceinline__ float elem_value(const float* chunk, int64_t nc, const float* ret, int64_t e)
{
    return e < nc ? chunk[e] : ret[e - nc];
}

// level 0: bins of bits [31:20] of every value; level 1: bins of bits [19:8] of the
// values whose bits [31:20] equal st->prefix1
__global__ void __launch_bounds__(kHistThreads)
k_sel_hist(const float* __restrict__ chunk, int64_t nc, const float* __restrict__ ret, int64_t nr, int level,
           SelState* __restrict__ st)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ unsigned h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kHistThreads) h[i] = 0;
    __syncthreads();
    const int64_t N = nc + nr;
    const unsigned p1 = st->prefix1;
    const int64_t stride = (int64_t)gridDim.x * kHistThreads;
    for (int64_t base = (int64_t)blockIdx.x * kHistThreads; base < N; base += stride) {
        const int64_t e = base + threadIdx.x;
        bool take = false;
        unsigned dig = 0;
        if (e < N) {
            const uint32_t b = __float_as_uint(elem_value(chunk, nc, ret, e));
            if (level == 0) { take = true; dig = b >> 20; }
            else { take = (b >> 20) == p1; dig = (b >> 8) & (kBins - 1); }
        }
        const unsigned key = take ? dig : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, key);
        if (take && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[dig], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += kHistThreads)
        if (h[i]) atomicAdd(&st->hist[level][i], h[i]);
}

// One CTA of SNT threads: the bin of histogram `level` that holds rank st->krem.
// After level 1 it forms the cut. The other histogram is cleared for reuse.
__global__ void __launch_bounds__(SNT) k_sel_scan(SelState* __restrict__ st, int level, CutParams cp)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ int ws[33];
    const unsigned* h = st->hist[level];
    const int b0 = 4 * threadIdx.x;
    const int h0 = (int)h[b0], h1 = (int)h[b0 + 1], h2 = (int)h[b0 + 2], h3 = (int)h[b0 + 3];
    const long long k = st->krem;
    int tot;
    const int excl = block_scan_excl(h0 + h1 + h2 + h3, ws, &tot);
    long long c = excl;
    const int hs[4] = {h0, h1, h2, h3};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (c < k && k <= c + hs[q]) {
            if (level == 0) { st->prefix1 = (unsigned)(b0 + q); st->krem = k - c; }
            else { st->prefix2 = (unsigned)(b0 + q); st->krem = k - c; }
        }
        c += hs[q];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += SNT) st->hist[1 - level][i] = 0;
    if (level == 1 && threadIdx.x == 0) {
        const uint32_t up_bits = (st->prefix1 << 20) | (st->prefix2 << 8) | 0xFFu;
        const float mup = __uint_as_float(up_bits);
        const double T = (double)mup + band_value(cp.lin, cp.quad, cp.rel, cp.safety, (double)mup);
        const float v = largest_v_below(cp, T, up_bits);
        st->cut = fminf(v, st->cut);
    }
}

// Keep the retained entries and chunk entries with M_hat <= cut (order not preserved:
// the final ordering sorts by (M64, draw index)).
__global__ void __launch_bounds__(kHistThreads)
k_sel_compact(const float* __restrict__ chunk, int64_t nc, uint64_t first, const float* __restrict__ rm_in,
              const uint64_t* __restrict__ ri_in, int64_t nr, SelState* __restrict__ st, float* __restrict__ rm_out,
              uint64_t* __restrict__ ri_out, int64_t cap_out)
{
    pdl_wait();
    pdl_launch_dependents();
    const float cut = st->cut;
    const int64_t N = nc + nr;
    const int64_t stride = (int64_t)gridDim.x * kHistThreads;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * kHistThreads; base < N; base += stride) {
        const int64_t e = base + threadIdx.x;
        float v = 0.f;
        uint64_t idx = 0;
        bool keep = false;
        if (e < N) {
            if (e < nr) { v = rm_in[e]; idx = ri_in[e]; }
            else { v = chunk[e - nr]; idx = first + (uint64_t)(e - nr); }
            keep = v <= cut;
        }
        const unsigned m = __ballot_sync(kFull, keep);
        if (m == 0) continue;
        long long pos0 = 0;
        if (lane == 0) pos0 = (long long)atomicAdd((unsigned long long*)&st->kept, (unsigned long long)__popc(m));
        pos0 = __shfl_sync(kFull, pos0, 0);
        if (keep) {
            const long long pos = pos0 + __popc(m & ((1u << lane) - 1u));
            if (pos < cap_out) { rm_out[pos] = v; ri_out[pos] = idx; }
        }
    }
}

// State of a new stream: the level-0 histogram cleared (each scan clears the other level for
// its next use), the cut, the counters and the end-of-stream fields (boundary M64 = NaN until
// the summary finds them). One launch instead of a memset and host-to-device copies.
__global__ void __launch_bounds__(SNT) k_sel_init(SelState* __restrict__ st, float cut)
{
    for (int i = threadIdx.x; i < kBins; i += SNT) st->hist[0][i] = 0;
    if (threadIdx.x == 0) {
        st->prefix1 = st->prefix2 = 0;
        st->krem = 0;
        st->cut = cut;
        st->kept = 0;
        st->nsel = 0;
        st->boundary[0] = st->boundary[1] = __longlong_as_double(0x7FF8000000000000ll);
        st->max_rel = st->max_over_band = st->thr = 0.0;
        st->violations = 0;
    }
}

__global__ void k_sel_begin(SelState* __restrict__ st, long long K)
{
    pdl_wait();
    pdl_launch_dependents();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->krem = K;
        st->kept = 0;
    }
}

// ---------------------------------------------------------------- ordering --
// rank_c = #{c' : (M64_c', idx_c') < (M64_c, idx_c)}, one warp per entry. M64 >= 0, so
// the order of the values is the order of their bit patterns as integers (no FP64 compares).
__global__ void k_rank(const double* __restrict__ m, const uint64_t* __restrict__ idx, int64_t r_host,
                       const long long* __restrict__ r_dev, int* __restrict__ rank)
{
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = r_dev ? (*r_dev < r_host ? *r_dev : r_host) : r_host;  // within the buffers
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long* mb = reinterpret_cast<const long long*>(m);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < r; c += nw) {
        const long long mc = mb[c];
        const uint64_t ic = idx[c];
        int cnt = 0;
        for (int64_t k = lane; k < r; k += 32) {
            const long long mk = mb[k];
            cnt += (mk < mc || (mk == mc && idx[k] < ic)) ? 1 : 0;
        }
        cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
        if (lane == 0) rank[c] = cnt;
    }
}

// Selection of entry c from its rank (q mode: rank < K) or its M64 (threshold mode:
// M64 <= a); thr_bits is the bit pattern of a >= 0 (M64 >= 0 orders like its bits) or -1.
__device__ __forceinline__ bool entry_selected(int q_mode, int rank, long long K, long long mbits, long long thr_bits)
{
    return q_mode ? (rank < K) : (mbits <= thr_bits);
}

// Selected entries go to position #{selected c' : idx_c' < idx_c}, one warp per entry
// (the selection is re-derived from the ranks, so no flag array is needed).
__global__ void k_place_sel(const double* __restrict__ m, const uint64_t* __restrict__ idx, const int* __restrict__ rank,
                            int64_t r_host, const long long* __restrict__ r_dev, long long K, int q_mode,
                            long long thr_bits, uint64_t* __restrict__ keys_out, double* __restrict__ m_out)
{
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = r_dev ? (*r_dev < r_host ? *r_dev : r_host) : r_host;  // within the buffers
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long* mb = reinterpret_cast<const long long*>(m);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < r; c += nw) {
        if (!entry_selected(q_mode, rank[c], K, mb[c], thr_bits)) continue;
        const uint64_t ic = idx[c];
        int cnt = 0;
        for (int64_t k = lane; k < r; k += 32)
            cnt += (entry_selected(q_mode, rank[k], K, mb[k], thr_bits) && idx[k] < ic) ? 1 : 0;
        cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
        if (lane == 0) {
            keys_out[cnt] = ic;
            m_out[cnt] = m[c];
        }
    }
}

// One CTA: accepted count, the M64 of ranks K-1 and K, the largest accepted M64 and the
// band statistics of the re-checked draws (the SelTail fields).
__global__ void __launch_bounds__(SNT)
k_sel_summary(const double* __restrict__ m64, const int* __restrict__ rank, const float* __restrict__ mhat, int64_t r_host,
              const long long* __restrict__ r_dev, long long K, int q_mode, long long thr_bits, CutParams cp,
              SelState* __restrict__ st)
{
    pdl_wait();
    pdl_launch_dependents();
    const int64_t r = r_dev ? (*r_dev < r_host ? *r_dev : r_host) : r_host;  // within the buffers
    __shared__ long long s_thr[32];
    __shared__ float s_rel[32], s_band[32];
    __shared__ int s_viol[32], s_n[32];
    const long long* mb = reinterpret_cast<const long long*>(m64);
    float mrel = 0.f, mband = 0.f;
    long long thr = -1;
    int viol = 0, nsel = 0;
    for (int64_t c = threadIdx.x; c < r; c += SNT) {
        const int rk = rank[c];
        const long long bits = mb[c];
        const bool sel = entry_selected(q_mode, rk, K, bits, thr_bits);
        if (q_mode) {
            if (rk == K - 1) st->boundary[0] = m64[c];
            if (rk == K) st->boundary[1] = m64[c];
        }
        if (sel) {
            ++nsel;
            thr = bits > thr ? bits : thr;
        }
        // diagnostics only: FP32 is enough (and cheap on B300)
        const float a = mhat[c], mf = (float)m64[c];
        const float err = fabsf(a - mf);
        const float band = (float)cp.safety * ((float)cp.lin * sqrtf(fmaxf(a, 0.f)) + (float)cp.quad + (float)cp.rel * a);
        if (mf > 0.f) mrel = fmaxf(mrel, __fdividef(err, mf));
        if (band > 0.f) mband = fmaxf(mband, __fdividef(err, band));
        viol += (err > band) ? 1 : 0;
    }
    for (int off = 16; off >= 1; off >>= 1) {
        mrel = fmaxf(mrel, __shfl_xor_sync(kFull, mrel, off));
        mband = fmaxf(mband, __shfl_xor_sync(kFull, mband, off));
        const long long o = __shfl_xor_sync(kFull, thr, off);
        thr = o > thr ? o : thr;
        viol += __shfl_xor_sync(kFull, viol, off);
        nsel += __shfl_xor_sync(kFull, nsel, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_rel[warp] = mrel; s_band[warp] = mband; s_thr[warp] = thr; s_viol[warp] = viol; s_n[warp] = nsel; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < SNT / 32; ++w) {
            mrel = fmaxf(mrel, s_rel[w]); mband = fmaxf(mband, s_band[w]); thr = s_thr[w] > thr ? s_thr[w] : thr;
            viol += s_viol[w]; nsel += s_n[w];
        }
        st->nsel = nsel;
        st->max_rel = mrel;
        st->max_over_band = mband;
        st->thr = thr >= 0 ? __longlong_as_double(thr) : -INFINITY;
        st->violations = viol;
    }
}

// grid of a grid-stride warp-per-item kernel: enough 256-thread CTAs for `count` warps,
// at most 16 per SM
unsigned warp_grid(const frr_ctx* ctx, uint64_t count)
{
    const uint64_t want = (count * 32 + 255) / 256;
    const uint64_t cap = (uint64_t)ctx->num_sms * 16;
    return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

template <int KB>
frr_status launch_bits_kb(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t count,
                          const long long* count_dev, const uint64_t* draws, uint32_t* rows)
{
    FRR_CUDA_TRY(ctx, launch_pdl(k_bits<KB>, warp_grid(ctx, count), 256, 0, ctx->stream, seed, exact ? 1 : 0, ctx->binom,
                                 (int)ctx->n, (int)ctx->n1, first, count, count_dev, draws, rows));
    return FRR_OK;
}

template <int KB>
frr_status launch_recheck_kb(frr_ctx* ctx, uint64_t seed, bool exact, const uint64_t* draws, int64_t count,
                             double* part, int ncb)
{
    dim3 grid((unsigned)((count + RG - 1) / RG), (unsigned)ncb);
    k_recheck<KB><<<grid, RCOLS, 0, ctx->stream>>>(ctx->Q, ctx->Qsum, ctx->qexp, (int)ctx->d, ctx->kused, (int)ctx->n,
                                                   (int)ctx->n1, seed, exact ? 1 : 0, ctx->binom, draws, count, part, ncb);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

}  // namespace

frr_status bits_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t count,
                       const uint64_t* draws, uint32_t* rows, const long long* count_dev)
{
    if (count == 0) return FRR_OK;
    switch (ctx->kb) {
        case 1: return launch_bits_kb<1>(ctx, seed, exact, first, count, count_dev, draws, rows);
        case 2: return launch_bits_kb<2>(ctx, seed, exact, first, count, count_dev, draws, rows);
        case 4: return launch_bits_kb<4>(ctx, seed, exact, first, count, count_dev, draws, rows);
        case 8: return launch_bits_kb<8>(ctx, seed, exact, first, count, count_dev, draws, rows);
        case 16: return launch_bits_kb<16>(ctx, seed, exact, first, count, count_dev, draws, rows);
        default: return FRR_E_UNSUPPORTED;
    }
}

frr_status words_select_launch(frr_ctx* ctx, const uint32_t* words, uint32_t* row)
{
    const int n = (int)ctx->n, n1 = (int)ctx->n1;
    switch (ctx->kb) {
        case 1: k_words_select<1><<<1, 32, 0, ctx->stream>>>(words, n, n1, row); break;
        case 2: k_words_select<2><<<1, 32, 0, ctx->stream>>>(words, n, n1, row); break;
        case 4: k_words_select<4><<<1, 32, 0, ctx->stream>>>(words, n, n1, row); break;
        case 8: k_words_select<8><<<1, 32, 0, ctx->stream>>>(words, n, n1, row); break;
        case 16: k_words_select<16><<<1, 32, 0, ctx->stream>>>(words, n, n1, row); break;
        default: return FRR_E_UNSUPPORTED;
    }
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

frr_status unpack_launch(frr_ctx* ctx, const uint32_t* rows, uint64_t count, uint8_t* w)
{
    if (count == 0) return FRR_OK;
    const uint64_t tot = count * (uint64_t)ctx->n;
    k_unpack<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(rows, 4 * ctx->kb, count, (int)ctx->n, w);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

frr_status recheck_sum_launch(frr_ctx* ctx, const double* part, int ncb, int64_t count, double* M64, double scale,
                              double denom, const long long* count_dev)
{
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(count, 256), 4 * ctx->num_sms));
    FRR_CUDA_TRY(ctx, launch_pdl(k_recheck_sum, grid, 256, 0, ctx->stream, part, ncb, count, count_dev, scale, denom,
                                 M64));
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

// The recheck of the selection path and of frr_recheck: the tensor-core digit-plane kernel.
frr_status recheck_launch(frr_ctx* ctx, uint64_t seed, bool exact, const uint64_t* draws, int64_t count, double* M64,
                          const long long* count_dev)
{
    return recheck_tc_launch(ctx, seed, exact, draws, count, M64, count_dev);
}

frr_status balance_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout)
{
    if (ctx->opts.precision == FRR_F32) return balance_f32_launch(ctx, seed, exact, first, B, Mout);
    return balance_tc_launch(ctx, seed, exact, first, B, Mout);
}

// ------------------------------------------------------------- streaming --
namespace {
constexpr uint64_t kChunkMax = 1ull << 22;

CutParams cut_params(const frr_ctx* ctx)
{
    const BandConsts& b = band_of(ctx);
    return CutParams{b.lin, b.quad, b.rel, ctx->opts.band_safety};
}

frr_status ensure_retained(frr_ctx* ctx, int which, int64_t entries)
{
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->ret_idx[which]), &ctx->ret_bytes_idx[which],
                          (size_t)entries * sizeof(uint64_t)));
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->ret_m[which]), &ctx->ret_bytes_m[which],
                          (size_t)entries * sizeof(float)));
    return FRR_OK;
}

double host_lower_bound(const frr_ctx* ctx, float v)
{
    const BandConsts& b = band_of(ctx);
    return (double)v - band_value(b.lin, b.quad, b.rel, ctx->opts.band_safety, (double)v);
}

float host_threshold_cut(const frr_ctx* ctx, double a)
{
    // largest float v >= 0 with L(v) <= a; {v : L(v) <= a} is an interval [0, v*] for a >= L(0)
    if (!(a < INFINITY)) return INFINITY;
    uint32_t lo = 0, hi = 0x7f800000u;
    float flo; memcpy(&flo, &lo, 4);
    if (host_lower_bound(ctx, flo) > a) return -1.0f;  // a < L(0): nothing can pass
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        float f; memcpy(&f, &mid, 4);
        if (host_lower_bound(ctx, f) <= a) lo = mid; else hi = mid;
    }
    float r; memcpy(&r, &lo, 4);
    return r;
}
}  // namespace

frr_status stream_begin(frr_ctx* ctx, uint64_t seed, double q, double threshold, uint64_t total)
{
    StreamState& st = ctx->st;
    st = StreamState{};
    st.active = true;
    st.exact = (seed == FRR_EXACT_SEED);
    st.seed = seed;
    st.q_mode = !isnan(q);
    st.q = q;
    st.threshold = threshold;
    st.total = total;
    if (st.q_mode) {
        const double qb = q * (double)total;
        double k = ceil(qb - 1e-9 * qb);
        if (k < 1.0) k = 1.0;
        if (k > (double)total) k = (double)total;
        st.K = (int64_t)k;
        st.cut = INFINITY;
    } else {
        st.K = 0;
        st.cut = host_threshold_cut(ctx, threshold);
    }
    st.retained = 0;
    ctx->ret_cur = 0;
    const double ms_init = ctx->stats.ms_init;
    FRR_TRY(ensure_device(ctx, &ctx->sel, &ctx->sel_bytes, sizeof(SelState)));
    k_sel_init<<<1, SNT, 0, ctx->stream>>>(static_cast<SelState*>(ctx->sel), st.cut);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.ms_init = ms_init;
    ctx->stats.boundary_gap_rel = NAN;
    return FRR_OK;
}

// Selection step over the approximate M of draws [first, first + bc) held in Mhat (device).
frr_status stream_select_step(frr_ctx* ctx, uint64_t first, uint64_t bc, const float* Mhat, bool last)
{
    StreamState& st = ctx->st;
    SelState* sel = static_cast<SelState*>(ctx->sel);
    const CutParams cp = cut_params(ctx);
    FRR_TRY(ensure_host_pinned(ctx, 256));
    const int in = ctx->ret_cur, out = 1 - in;
    const int64_t N = st.retained + (int64_t)bc;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, kHistThreads), 4 * ctx->num_sms));
    FRR_CUDA_TRY(ctx, launch_pdl(k_sel_begin, 1, 32, 0, ctx->stream, sel, (long long)st.K));
    if (st.q_mode && N > st.K) {
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_hist, grid, kHistThreads, 0, ctx->stream, Mhat, (int64_t)bc, ctx->ret_m[in],
                                     st.retained, 0, sel));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_scan, 1, SNT, 0, ctx->stream, sel, 0, cp));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_hist, grid, kHistThreads, 0, ctx->stream, Mhat, (int64_t)bc, ctx->ret_m[in],
                                     st.retained, 1, sel));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_scan, 1, SNT, 0, ctx->stream, sel, 1, cp));
    }
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    int64_t cap = (int64_t)(ctx->ret_bytes_m[out] / sizeof(float));
    // the last chunk of a deferred-count stream keeps every entry it could keep (capacity N),
    // so the count need not be read back before the recheck
    const bool defer = last && st.defer_count && N <= (int64_t)(1 << 20);
    // Deferred (count not read back): in q mode the retained set is about K plus the draws
    // inside the band around the cut, so 4 K + 16384 entries hold it; a larger set overflows
    // the buffer, which stream_end detects (the count is read back there) and the caller then
    // redoes the selection without deferral. Threshold mode keeps room for every draw.
    const int64_t want = defer ? (st.q_mode ? std::min<int64_t>(N, 4 * st.K + 16384) : N)
                               : std::min<int64_t>(N, std::max<int64_t>(4 * st.K + 65536, 1 << 20));
    if (cap < want) {
        FRR_TRY(ensure_retained(ctx, out, want));
        cap = (int64_t)(ctx->ret_bytes_m[out] / sizeof(float));
    }
    if (defer) {
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_compact, grid, kHistThreads, 0, ctx->stream, Mhat, (int64_t)bc, first,
                                     ctx->ret_m[in], ctx->ret_idx[in], st.retained, sel, ctx->ret_m[out],
                                     ctx->ret_idx[out], cap));
        FRR_CUDA_TRY(ctx, cudaGetLastError());
        if (st.timing) cudaEventRecord(ctx->ev[2], ctx->stream);
        st.retained = -1;
        st.retained_bound = std::min<int64_t>(N, cap);
        ctx->ret_cur = out;
        return FRR_OK;
    }
    for (int attempt = 0;; ++attempt) {
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_compact, grid, kHistThreads, 0, ctx->stream, Mhat, (int64_t)bc, first,
                                     ctx->ret_m[in], ctx->ret_idx[in], st.retained, sel, ctx->ret_m[out],
                                     ctx->ret_idx[out], cap));
        FRR_CUDA_TRY(ctx, cudaGetLastError());
        long long* hk = static_cast<long long*>(ctx->host_pinned);
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk, &sel->kept, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk + 1, ctx->dev_counters + 12, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        if (st.timing) cudaEventRecord(ctx->ev[2], ctx->stream);
        FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        const long long kept = hk[0];
        if (*reinterpret_cast<int*>(hk + 1) != 0) {
            FRR_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dev_counters + 12, 0, sizeof(int), ctx->stream));
            FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            return FRR_E_TIMEOUT;
        }
        if (kept <= cap) {
            st.retained = kept;
            break;
        }
        if (attempt == 1) return FRR_E_CAPACITY;
        // the cut stays as computed, so the re-run keeps the same set
        FRR_TRY(ensure_retained(ctx, out, kept));
        cap = (int64_t)(ctx->ret_bytes_m[out] / sizeof(float));
        k_sel_begin<<<1, 32, 0, ctx->stream>>>(sel, st.K);
    }
    ctx->ret_cur = out;
    return FRR_OK;
}

frr_status stream_chunk(frr_ctx* ctx, uint64_t first, uint64_t B)
{
    StreamState& st = ctx->st;
    if (!st.active) return FRR_E_STATE;
    if (B == 0) return FRR_OK;
    if (st.seen + B > st.total) return FRR_E_RANGE;
    for (uint64_t off = 0; off < B; off += kChunkMax) {
        const uint64_t bc = std::min<uint64_t>(kChunkMax, B - off);
        FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->Mhat), &ctx->Mhat_bytes, bc * sizeof(float)));
        if (st.timing) cudaEventRecord(ctx->ev[0], ctx->stream);
        FRR_TRY(balance_launch(ctx, st.seed, st.exact, first + off, bc, ctx->Mhat));
        if (st.timing) cudaEventRecord(ctx->ev[1], ctx->stream);
        FRR_TRY(stream_select_step(ctx, first + off, bc, ctx->Mhat, st.seen + off + bc == st.total));
        if (st.retained < 0) {
            st.times_pending = true;  // nothing was synchronised: read the events in stream_end
            continue;
        }
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&t2, ctx->ev[1], ctx->ev[2]);
        ctx->stats.ms_balance += t1;
        ctx->stats.ms_select += t2;
    }
    st.seen += B;
    ctx->stats.draws += (int64_t)B;
    return FRR_OK;
}

// Selection over draws whose approximate M was computed elsewhere (the batched launch).
frr_status stream_chunk_precomputed(frr_ctx* ctx, uint64_t first, uint64_t B, const float* Mhat)
{
    StreamState& st = ctx->st;
    if (!st.active) return FRR_E_STATE;
    if (st.seen + B > st.total) return FRR_E_RANGE;
    for (uint64_t off = 0; off < B; off += kChunkMax) {
        const uint64_t bc = std::min<uint64_t>(kChunkMax, B - off);
        if (st.timing) cudaEventRecord(ctx->ev[0], ctx->stream);  // no balance here: an empty interval
        if (st.timing) cudaEventRecord(ctx->ev[1], ctx->stream);
        FRR_TRY(stream_select_step(ctx, first + off, bc, Mhat + off, st.seen + off + bc == st.total));
        if (st.retained < 0) {
            st.times_pending = st.timing;  // nothing was synchronised: read the events in stream_end
            continue;
        }
        float t2 = 0.f;
        if (st.timing) cudaEventElapsedTime(&t2, ctx->ev[1], ctx->ev[2]);
        ctx->stats.ms_select += t2;
    }
    st.seen += B;
    ctx->stats.draws += (int64_t)B;
    return FRR_OK;
}

frr_status stream_end_enqueue(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, size_t extra_pinned)
{
    StreamState& st = ctx->st;
    if (!st.active || st.end_enqueued) return FRR_E_STATE;
    if (st.seen != st.total) return FRR_E_STATE;
    // the retained count is either known on the host, or (deferred) only on the device,
    // bounded by retained_bound: the kernels below then read it there
    const bool dev_count = st.retained < 0;
    const int64_t rb = dev_count ? st.retained_bound : st.retained;
    const int cur = ctx->ret_cur;
    SelState* sel = static_cast<SelState*>(ctx->sel);
    const long long* r_dev = dev_count ? &sel->kept : nullptr;
    // Where the accepted keys go. q mode accepts exactly K draws, so when K fits the
    // placement kernel writes them straight into device outputs; host outputs are copied
    // into pinned memory together with the summary (the first min(cap, r) entries hold them
    // whenever they fit). Either way one synchronisation serves the call.
    const bool host_keys = cap > 0 && !is_device_ptr(keys_out);
    const bool host_m = M64_out != nullptr && cap > 0 && !is_device_ptr(M64_out);
    const bool direct = st.q_mode && st.K <= cap && !host_keys && !host_m;
    const int64_t stage_n = std::min<int64_t>(cap, rb);
    const bool stage = !direct && (host_keys || host_m) && stage_n > 0;
    const size_t used = 256 + (stage ? (size_t)stage_n * 16 : 0);
    FRR_TRY(ensure_host_pinned(ctx, used + extra_pinned));
    st.end_enqueued = true;
    st.end_direct = direct;
    st.end_host_keys = host_keys;
    st.end_host_m = host_m;
    st.end_stage = stage;
    st.end_dev_count = dev_count;
    st.end_rb = rb;
    st.end_stage_n = stage_n;
    st.end_pinned = used;
    if (st.timing) cudaEventRecord(ctx->ev[3], ctx->stream);
    // scratch: M64 (r), M64 out (r), keys out (r), rank (r)
    const size_t need = (size_t)rb * (3 * sizeof(double) + sizeof(int)) + 64;
    FRR_TRY(ensure_device(ctx, &ctx->misc, &ctx->misc_bytes, need));
    char* base = static_cast<char*>(ctx->misc);
    double* m64 = reinterpret_cast<double*>(base);
    double* mout = m64 + rb;
    uint64_t* kout = reinterpret_cast<uint64_t*>(mout + rb);
    int* rank = reinterpret_cast<int*>(kout + rb);
    char* hp = static_cast<char*>(ctx->host_pinned);
    uint64_t* hk = reinterpret_cast<uint64_t*>(hp + 256);
    double* hm = reinterpret_cast<double*>(hk + stage_n);
    uint64_t* place_k = direct ? keys_out : kout;
    double* place_m = (direct && M64_out) ? M64_out : mout;
    if (rb > 0) {
        // (sel->boundary was set to NaN by k_sel_init)
        FRR_TRY(recheck_launch(ctx, st.seed, st.exact, ctx->ret_idx[cur], rb, m64, r_dev));
        // threshold mode: M64 <= a compares as bit patterns (M64 >= 0); a < 0 accepts nothing
        long long thr_bits = -1;
        if (!st.q_mode && st.threshold >= 0.0) memcpy(&thr_bits, &st.threshold, sizeof(thr_bits));
        FRR_CUDA_TRY(ctx, launch_pdl(k_rank, warp_grid(ctx, rb), 256, 0, ctx->stream, m64, ctx->ret_idx[cur], rb, r_dev,
                                     rank));
        FRR_CUDA_TRY(ctx, launch_pdl(k_place_sel, warp_grid(ctx, rb), 256, 0, ctx->stream, m64, ctx->ret_idx[cur], rank,
                                     rb, r_dev, (long long)st.K, st.q_mode ? 1 : 0, thr_bits, place_k, place_m));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_summary, 1, SNT, 0, ctx->stream, m64, rank, ctx->ret_m[cur], rb, r_dev,
                                     (long long)st.K, st.q_mode ? 1 : 0, thr_bits, cut_params(ctx), sel));
        FRR_CUDA_TRY(ctx, cudaGetLastError());
        // kept (the retained count) and the SelTail fields, in one copy
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hp, &sel->kept, sizeof(long long) + sizeof(SelTail), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hp + 128, ctx->dev_counters + 12, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        if (stage) {
            if (host_keys)
                FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk, kout, (size_t)stage_n * 8, cudaMemcpyDeviceToHost, ctx->stream));
            if (host_m)
                FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hm, mout, (size_t)stage_n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    if (st.timing) cudaEventRecord(ctx->ev[4], ctx->stream);
    return FRR_OK;
}

const uint64_t* stream_end_keys_dev(const frr_ctx* ctx, const uint64_t* keys_out)
{
    if (ctx->st.end_direct) return keys_out;
    const double* m64 = static_cast<const double*>(ctx->misc);
    return reinterpret_cast<const uint64_t*>(m64 + 2 * ctx->st.end_rb);
}

size_t stream_end_pinned_used(const frr_ctx* ctx) { return ctx->st.end_pinned; }

size_t stream_end_pinned_bound(const frr_ctx* ctx, int64_t cap)
{
    // the staged outputs hold min(cap, retained) entries of 16 bytes; a deferred q-mode
    // stream retains at most its buffer's capacity, 4 K + 16384 entries grown by a quarter
    // (ensure_device)
    const StreamState& st = ctx->st;
    int64_t rb = (int64_t)st.total;
    if (st.q_mode) rb = std::min<int64_t>(rb, (4 * st.K + 16384) + (4 * st.K + 16384) / 4 + 1);
    return 256 + (size_t)std::max<int64_t>(0, std::min<int64_t>(cap, rb)) * 16;
}

frr_status stream_end_finish(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out)
{
    StreamState& st = ctx->st;
    if (!st.active || !st.end_enqueued) return FRR_E_STATE;
    st.end_enqueued = false;
    const int64_t rb = st.end_rb;
    const bool direct = st.end_direct, host_keys = st.end_host_keys, host_m = st.end_host_m;
    const int64_t stage_n = st.end_stage_n;
    double* m64 = static_cast<double*>(ctx->misc);
    double* mout = m64 + rb;
    uint64_t* kout = reinterpret_cast<uint64_t*>(mout + rb);
    char* hp = static_cast<char*>(ctx->host_pinned);
    uint64_t* hk = reinterpret_cast<uint64_t*>(hp + 256);
    double* hm = reinterpret_cast<double*>(hk + stage_n);
    SelTail tail{};
    tail.boundary[0] = tail.boundary[1] = NAN;
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t r = rb;
    if (rb > 0) {
        if (st.end_dev_count) memcpy(&r, hp, sizeof(long long));
        memcpy(&tail, hp + sizeof(long long), sizeof(SelTail));
        if (*reinterpret_cast<int*>(hp + 128) != 0) {
            FRR_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dev_counters + 12, 0, sizeof(int), ctx->stream));
            FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            st.active = false;
            return FRR_E_TIMEOUT;
        }
        if (r > rb) {
            // the deferred retained set outgrew its buffer: nothing written; redo undeferred
            st.active = false;
            st.overflowed = true;
            return FRR_E_CAPACITY;
        }
    }
    if (st.times_pending) {
        float t1 = 0.f, t2 = 0.f;
        cudaEventElapsedTime(&t1, ctx->ev[0], ctx->ev[1]);
        cudaEventElapsedTime(&t2, ctx->ev[1], ctx->ev[2]);
        ctx->stats.ms_balance += t1;
        ctx->stats.ms_select += t2;
        st.times_pending = false;
    }
    float t = 0.f;
    if (st.timing) cudaEventElapsedTime(&t, ctx->ev[3], ctx->ev[4]);
    ctx->stats.ms_recheck += t;
    const long long nsel = tail.nsel;
    *K_out = nsel;
    st.active = false;
    st.retained = r;

    const BandConsts& b = band_of(ctx);
    ctx->stats.candidates = r;
    ctx->stats.accepted = nsel;
    ctx->stats.max_rel_err = tail.max_rel;
    ctx->stats.max_err_over_band = tail.max_over_band;
    ctx->stats.band_violations = tail.violations;
    ctx->stats.threshold_m64 = nsel > 0 ? tail.thr : NAN;
    ctx->stats.band_at_threshold = nsel > 0 ? band_value(b.lin, b.quad, b.rel, ctx->opts.band_safety, tail.thr) : NAN;
    if (st.q_mode && !isnan(tail.boundary[0]) && !isnan(tail.boundary[1])) {
        ctx->stats.boundary_gap_rel = (tail.boundary[1] - tail.boundary[0]) / tail.boundary[0];
        ctx->stats.parity_at_risk = ctx->stats.boundary_gap_rel < 1e-11 ? 1 : 0;
    }
    if (nsel > cap) return FRR_E_CAPACITY;
    if (nsel > 0 && !direct) {
        bool device_copies = false;
        if (host_keys) {
            memcpy(keys_out, hk, (size_t)nsel * sizeof(uint64_t));
        } else {
            FRR_CUDA_TRY(ctx, cudaMemcpyAsync(keys_out, kout, (size_t)nsel * sizeof(uint64_t), cudaMemcpyDefault,
                                              ctx->stream));
            device_copies = true;
        }
        if (M64_out) {
            if (host_m) {
                memcpy(M64_out, hm, (size_t)nsel * sizeof(double));
            } else {
                FRR_CUDA_TRY(ctx, cudaMemcpyAsync(M64_out, mout, (size_t)nsel * sizeof(double), cudaMemcpyDefault,
                                                  ctx->stream));
                device_copies = true;
            }
        }
        if (device_copies) FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return FRR_OK;
}

frr_status stream_end(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out)
{
    FRR_TRY(stream_end_enqueue(ctx, keys_out, M64_out, cap, 0));
    return stream_end_finish(ctx, keys_out, M64_out, cap, K_out);
}

}  // namespace frr

namespace frr {

// The int64 CUDA-core form of the recheck (the same exact treated sums as the tensor-core
// form behind recheck_launch) with the per-CTA partial sums in a device array the caller
// provides (part_capacity doubles); nothing is allocated. Pool seeds only.
frr_status recheck_launch_into(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count, double* part,
                               size_t part_capacity, double* M64)
{
    if (count <= 0) return FRR_OK;
    const int ncb = ceil_div(ctx->d, RCOLS);
    if ((size_t)count * (size_t)ncb > part_capacity) return FRR_E_CAPACITY;
    frr_status s;
    switch (ctx->kb) {
        case 1: s = launch_recheck_kb<1>(ctx, seed, false, draws, count, part, ncb); break;
        case 2: s = launch_recheck_kb<2>(ctx, seed, false, draws, count, part, ncb); break;
        case 4: s = launch_recheck_kb<4>(ctx, seed, false, draws, count, part, ncb); break;
        case 8: s = launch_recheck_kb<8>(ctx, seed, false, draws, count, part, ncb); break;
        case 16: s = launch_recheck_kb<16>(ctx, seed, false, draws, count, part, ncb); break;
        default: return FRR_E_UNSUPPORTED;
    }
    FRR_TRY(s);
    const double scale = ((double)ctx->n1 * (double)ctx->n0) / (double)ctx->n;
    k_recheck_sum<<<ceil_div(count, 256), 256, 0, ctx->stream>>>(part, ncb, count, nullptr, scale, 1.0, M64);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

}  // namespace frr

// ------------------------------------------------------ stream checkpoints --
// A stream between chunks is fully described by its parameters, the cut on the approximate
// M and the retained set (draw index, approximate M); key-only storage (Sec. 2.1) keeps it
// small. The blob is a 256-byte header followed by the retained indices (uint64) and their
// approximate M (float), little-endian; its FNV-1a checksum covers everything else.
namespace frr {
namespace {

constexpr char kBlobMagic[8] = {'F', 'R', 'R', 'S', 'T', 'R', 'M', '\0'};
constexpr uint32_t kBlobVersion = 1;
constexpr size_t kBlobHeader = 256;

struct BlobHeader {               // 256 bytes
    char magic[8];
    uint32_t version, header_bytes;
    int64_t n, d, n1;
    int32_t precision, whiten;
    double ridge, band_safety;
    double band_lin, band_quad, band_rel;
    uint64_t seed, total, seen;
    int32_t exact, q_mode;
    double q, threshold;
    int64_t K, retained;
    float cut;
    uint32_t pad0;
    int64_t stat_draws;
    double stat_ms_balance, stat_ms_select;
    unsigned char reserved[64];
    uint64_t checksum;
};
static_assert(sizeof(BlobHeader) == kBlobHeader, "stream checkpoint header layout");
static_assert(offsetof(BlobHeader, checksum) == 248, "stream checkpoint header layout");

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes)
{
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= c[i];
        h *= 0x100000001B3ull;
    }
    return h;
}

uint64_t blob_checksum(const BlobHeader& h, const void* payload, size_t payload_bytes)
{
    BlobHeader z = h;
    z.checksum = 0;
    const uint64_t h0 = fnv1a(0xCBF29CE484222325ull, &z, sizeof(z));
    return fnv1a(h0, payload, payload_bytes);
}

}  // namespace

frr_status stream_blob_check(const void* blob, size_t size, frr_stream_info* info)
{
    if (!blob || size < kBlobHeader) return FRR_E_ARG;
    BlobHeader h;
    memcpy(&h, blob, sizeof(h));
    if (memcmp(h.magic, kBlobMagic, sizeof(kBlobMagic)) != 0) return FRR_E_ARG;
    if (h.version != kBlobVersion || h.header_bytes != kBlobHeader) return FRR_E_UNSUPPORTED;
    if (h.retained < 0 || h.retained > (int64_t)((size - kBlobHeader) / 12) ||
        size != kBlobHeader + (size_t)h.retained * 12)
        return FRR_E_ARG;
    if (blob_checksum(h, static_cast<const char*>(blob) + kBlobHeader, size - kBlobHeader) != h.checksum)
        return FRR_E_ARG;
    if (h.seen > h.total || h.n < 2 || h.d < 1 || h.n1 < 1 || h.n1 > h.n - 1) return FRR_E_ARG;
    if (info) {
        info->version = (int32_t)h.version;
        info->n = h.n;
        info->d = h.d;
        info->n1 = h.n1;
        info->precision = h.precision;
        info->seed = h.seed;
        info->total = h.total;
        info->seen = h.seen;
        info->q = h.q;
        info->threshold = h.threshold;
        info->K = h.K;
        info->retained = h.retained;
    }
    return FRR_OK;
}

frr_status stream_save(frr_ctx* ctx, void* blob, size_t cap, size_t* size_out)
{
    StreamState& st = ctx->st;
    if (!st.active || st.end_enqueued || st.retained < 0) return FRR_E_STATE;
    const size_t size = kBlobHeader + (size_t)st.retained * 12;
    *size_out = size;
    if (!blob || cap < size) return FRR_E_CAPACITY;
    BlobHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kBlobMagic, sizeof(kBlobMagic));
    h.version = kBlobVersion;
    h.header_bytes = kBlobHeader;
    h.n = ctx->n;
    h.d = ctx->d;
    h.n1 = ctx->n1;
    h.precision = ctx->opts.precision;
    h.whiten = ctx->opts.whiten;
    h.ridge = ctx->opts.ridge;
    h.band_safety = ctx->opts.band_safety;
    const BandConsts& b = band_of(ctx);
    h.band_lin = b.lin;
    h.band_quad = b.quad;
    h.band_rel = b.rel;
    h.seed = st.seed;
    h.total = st.total;
    h.seen = st.seen;
    h.exact = st.exact ? 1 : 0;
    h.q_mode = st.q_mode ? 1 : 0;
    h.q = st.q;
    h.threshold = st.threshold;
    h.K = st.K;
    h.retained = st.retained;
    // the running cut lives on the device (each chunk's scan may tighten it)
    SelState* sel = static_cast<SelState*>(ctx->sel);
    float cut = st.cut;
    FRR_TRY(copy_out(ctx, &cut, &sel->cut, sizeof(float)));
    h.cut = cut;
    h.stat_draws = ctx->stats.draws;
    h.stat_ms_balance = ctx->stats.ms_balance;
    h.stat_ms_select = ctx->stats.ms_select;
    char* payload = static_cast<char*>(blob) + kBlobHeader;
    const int cur = ctx->ret_cur;
    if (st.retained > 0) {
        FRR_TRY(copy_out(ctx, payload, ctx->ret_idx[cur], (size_t)st.retained * sizeof(uint64_t)));
        FRR_TRY(copy_out(ctx, payload + (size_t)st.retained * sizeof(uint64_t), ctx->ret_m[cur],
                         (size_t)st.retained * sizeof(float)));
    }
    h.checksum = blob_checksum(h, payload, size - kBlobHeader);
    memcpy(blob, &h, sizeof(h));
    return FRR_OK;
}

frr_status stream_load(frr_ctx* ctx, const void* blob, size_t size)
{
    FRR_TRY(stream_blob_check(blob, size, nullptr));
    BlobHeader h;
    memcpy(&h, blob, sizeof(h));
    // the blob must come from a context that scores draws identically: same shape, options
    // and (through the covariates) the same error-band constants
    const BandConsts& b = band_of(ctx);
    if (h.n != ctx->n || h.d != ctx->d || h.n1 != ctx->n1 || h.precision != ctx->opts.precision ||
        h.whiten != ctx->opts.whiten || h.band_safety != ctx->opts.band_safety ||
        (ctx->opts.whiten == FRR_RIDGE && h.ridge != ctx->opts.ridge) || h.band_lin != b.lin || h.band_quad != b.quad ||
        h.band_rel != b.rel)
        return FRR_E_ARG;
    const bool exact = h.exact != 0;
    if (exact && (ctx->n > kExactMaxN || h.total > binom_host((int)ctx->n, (int)ctx->n1))) return FRR_E_ARG;
    FRR_TRY(stream_begin(ctx, h.seed, h.q_mode ? h.q : NAN, h.q_mode ? NAN : h.threshold, h.total));
    StreamState& st = ctx->st;
    if ((h.q_mode != 0) != st.q_mode || (st.q_mode && st.K != h.K)) {
        st.active = false;
        return FRR_E_ARG;
    }
    st.seen = h.seen;
    st.cut = h.cut;
    const char* payload = static_cast<const char*>(blob) + kBlobHeader;
    if (h.retained > 0) {
        frr_status s = ensure_retained(ctx, 0, h.retained);
        if (s == FRR_OK) s = copy_in(ctx, ctx->ret_idx[0], payload, (size_t)h.retained * sizeof(uint64_t));
        if (s == FRR_OK)
            s = copy_in(ctx, ctx->ret_m[0], payload + (size_t)h.retained * sizeof(uint64_t),
                        (size_t)h.retained * sizeof(float));
        if (s != FRR_OK) {
            st.active = false;
            return s;
        }
    }
    ctx->ret_cur = 0;
    st.retained = h.retained;
    // the device-side cut of the restored stream (stream_begin set the fresh one)
    SelState* sel = static_cast<SelState*>(ctx->sel);
    frr_status s = copy_in(ctx, &sel->cut, &h.cut, sizeof(float));
    if (s != FRR_OK) {
        st.active = false;
        return s;
    }
    ctx->stats.draws = h.stat_draws;
    ctx->stats.ms_balance = h.stat_ms_balance;
    ctx->stats.ms_select = h.stat_ms_select;
    return FRR_OK;
}

}  // namespace frr
