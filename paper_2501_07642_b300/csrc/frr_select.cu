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
                       uint32_t* __restrict__ rows, int* __restrict__ zero, int nzero)
{
    pdl_wait();
    pdl_launch_dependents();
    // counters of the kernel that follows (the recheck's per-tile completion counts)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nzero; i += gridDim.x * blockDim.x) zero[i] = 0;
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

// A cut for the upper edge m_up of the bin that holds the K-th smallest M_hat: every v with
// L(v) = v - band(v) <= T, T = U(m_up) = m_up + band(m_up), must be kept. L is increasing
// beyond its minimum near 0, and with x = sqrt(v), L(v) = T is the quadratic
// (1 - s rel) x^2 - s lin x - (s quad + T) = 0, band(v) = s (lin sqrt(v) + quad + rel v). The
// root is evaluated in FP32 with every operation rounded towards the larger result (and
// the leading coefficient rounded down, which can only enlarge the root), so the value
// returned is at or above the exact bound: a few more draws may be kept, never fewer.
__device__ float cut_upper_bound(const CutParams& cp, float mup)
{
    if (!(mup < INFINITY)) return INFINITY;
    const float s = __double2float_ru(cp.safety), lin = __double2float_ru(cp.lin);
    const float quad = __double2float_ru(cp.quad), rel = __double2float_ru(cp.rel);
    const float band = __fmul_ru(s, __fadd_ru(__fadd_ru(__fmul_ru(lin, __fsqrt_ru(mup)), quad), __fmul_ru(rel, mup)));
    const float T = __fadd_ru(mup, band);
    const float A = __fsub_rd(1.0f, __fmul_ru(s, rel));
    if (!(A > 0.0f)) return INFINITY;
    const float Bq = __fmul_ru(s, lin), Cq = __fadd_ru(__fmul_ru(s, quad), T);
    const float disc = __fadd_ru(__fmul_ru(Bq, Bq), __fmul_ru(__fmul_ru(4.0f, A), Cq));
    const float x = __fdiv_ru(__fadd_ru(Bq, __fsqrt_ru(disc)), __fmul_rd(2.0f, A));
    return fmaxf(__fmul_ru(x, x), mup);
}

// ---- cut and compaction over V = retained (nr values) + chunk (nc values)
// Two histogram levels on the float bit pattern (M_hat >= 0, so the bit order is the
// value order): bits [31:20] over all of V, then bits [19:8] inside the bin that holds
// the K-th smallest. The K-th smallest value lies below the upper edge m_up of the
// second-level bin, so T = U(m_up) >= U(M_(K)) is a safe cut; it is looser than the
// exact one by at most 2^-15 relative.
// The level-0 counts are kept per stream in one of two histogram sets (parity of the
// chunk): the split-BF16 balance kernel adds each chunk's values as it scores them (or
// k_sel_hist0 does), and the compaction of the previous chunk has added the values it
// kept. k_sel_level1 then finds the level-0 bin of rank K (every CTA reads the 4096 bins)
// and counts level 1; k_sel_keep forms the cut, compacts, and adds the kept values to the
// other set, which k_sel_level1 has cleared. Two launches per chunk, all SMs busy.
constexpr int kBins = 4096;
constexpr int kSelThreads = 512;
constexpr int kSelUnroll = 4;

struct SelState {
    unsigned hist0[2][kBins];  // level-0 counts, per chunk parity
    unsigned hist1[2][kBins];  // level-1 counts, per chunk parity
    unsigned p1;               // level-0 bin of rank K (k_sel_level1 -> k_sel_keep)
    int pad2;
    long long krem;            // rank K inside that bin
    float cut;
    int pad0;
    long long kept;
    // end-of-stream results, read back in one copy together with kept (see SelTail)
    long long nsel;
    double boundary[2];      // M64 of ranks K-1 and K (q mode)
    double max_rel, max_over_band, thr;
    int violations;
    int err;                 // the context's device error word once the selection has run
    int fin_overflow;        // more retained draws than the one-CTA finish holds: redo
    int pad1;
};

// the part of SelState read back by the host at the end of a stream (after kept)
struct SelTail {
    long long nsel;
    double boundary[2];
    double max_rel, max_over_band, thr;
    int violations;
    int err;
    int fin_overflow;
    int pad1;
};
static_assert(offsetof(SelState, nsel) - offsetof(SelState, kept) == sizeof(long long), "kept precedes the tail");
static_assert(offsetof(SelState, violations) - offsetof(SelState, nsel) == offsetof(SelTail, violations), "tail layout");
static_assert(offsetof(SelState, fin_overflow) - offsetof(SelState, nsel) == offsetof(SelTail, fin_overflow), "tail layout");
static_assert(sizeof(SelState) - offsetof(SelState, nsel) == sizeof(SelTail), "tail layout");

__device__ __forceinline__ float sel_elem(const float* ret, int64_t nr, const float* chunk, int64_t e)
{
    return e < nr ? ret[e] : chunk[e - nr];
}

// Adds 1 to bin `dig` of h for every lane with take, one atomic per distinct bin of the warp.
__device__ __forceinline__ void warp_count(unsigned* h, bool take, unsigned dig)
{
    const unsigned key = take ? dig : 0xffffffffu;
    const unsigned peers = __match_any_sync(kFull, key);
    if (take && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[dig], (unsigned)__popc(peers));
}

// Zeroes a shared histogram, and adds its non-zero bins to a global one afterwards.
__device__ __forceinline__ void shist_clear(unsigned* h)
{
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0u;
    __syncthreads();
}
__device__ __forceinline__ void shist_flush(const unsigned* h, unsigned* g)
{
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&g[i], h[i]);
}

// The bin of the global histogram g that holds rank k (1-based; k <= the total count), and
// k minus the counts of the bins before it. Every thread of the block gets the answer.
__device__ void find_bin(const unsigned* __restrict__ g, long long k, unsigned* bin_out, long long* k_out)
{
    __shared__ long long s_part[kSelThreads / 32];
    __shared__ unsigned s_bin;
    __shared__ long long s_k;
    constexpr int per = kBins / kSelThreads;  // 8 consecutive bins per thread
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint4 a = *reinterpret_cast<const uint4*>(g + per * tid);
    const uint4 b = *reinterpret_cast<const uint4*>(g + per * tid + 4);
    const unsigned c[per] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    long long mine = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) mine += c[i];
    long long incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_part[warp] = incl;
    __syncthreads();
    long long before = incl - mine;
    for (int w = 0; w < warp; ++w) before += s_part[w];
    if (before < k && k <= before + mine) {
        long long run = before;
#pragma unroll
        for (int i = 0; i < per; ++i) {
            if (run < k && k <= run + (long long)c[i]) {
                s_bin = (unsigned)(per * tid + i);
                s_k = k - run;
            }
            run += c[i];
        }
    }
    __syncthreads();
    *bin_out = s_bin;
    *k_out = s_k;
    __syncthreads();
}

// Level-0 counts of the values [0, nc) of a chunk into the global histogram g, for a chunk
// whose balance kernel did not add them (FP32 path, values computed elsewhere, a restored stream).
__global__ void __launch_bounds__(kSelThreads)
k_sel_hist0(const float* __restrict__ vals, int64_t nc, unsigned* __restrict__ g)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ unsigned h[kBins];
    shist_clear(h);
    const int64_t stride = (int64_t)gridDim.x * kSelThreads;
    for (int64_t base = (int64_t)blockIdx.x * kSelThreads; base < nc; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool take = e < nc;
        warp_count(h, take, take ? (__float_as_uint(vals[e]) >> 20) : 0u);
    }
    shist_flush(h, g);
}

// Grid of the selection kernels: one slice of V per CTA, at most one CTA per SM.
__host__ __device__ inline int64_t sel_slice(int64_t N, int grid) { return (N + grid - 1) / grid; }

// Level 1 of the cut (when new_cut) over V; also clears the other parity's histograms and the
// kept counter for k_sel_keep.
__global__ void __launch_bounds__(kSelThreads)
k_sel_level1(const float* __restrict__ ret_m, int64_t nr, const float* __restrict__ chunk, int64_t nc, long long K,
             int new_cut, int par, SelState* __restrict__ st)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ unsigned h[kBins];
    const int tid = threadIdx.x;
    // the other set was last read by the previous chunk's kernels, which have completed
    for (int i = blockIdx.x * kSelThreads + tid; i < kBins; i += gridDim.x * kSelThreads) {
        st->hist0[1 - par][i] = 0u;
        st->hist1[1 - par][i] = 0u;
    }
    if (blockIdx.x == 0 && tid == 0) st->kept = 0;
    if (!new_cut) return;
    unsigned p1;
    long long krem;
    find_bin(st->hist0[par], K, &p1, &krem);
    if (blockIdx.x == 0 && tid == 0) {
        st->p1 = p1;
        st->krem = krem;
    }
    shist_clear(h);
    const int64_t N = nr + nc, per = sel_slice(N, gridDim.x);
    const int64_t lo = std::min<int64_t>(N, (int64_t)blockIdx.x * per), hi = std::min<int64_t>(N, lo + per);
    for (int64_t base = lo; base < hi; base += (int64_t)kSelThreads * kSelUnroll) {
        float v[kSelUnroll];
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const int64_t e = base + (int64_t)u * kSelThreads + tid;
            v[u] = e < hi ? sel_elem(ret_m, nr, chunk, e) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const int64_t e = base + (int64_t)u * kSelThreads + tid;
            const uint32_t b = __float_as_uint(v[u]);
            warp_count(h, e < hi && (b >> 20) == p1, (b >> 8) & (kBins - 1));
        }
    }
    shist_flush(h, st->hist1[par]);
}

// The cut (when new_cut: from the level-1 counts, looser than the exact K-th value by at
// most 2^-15 relative plus the directed rounding of cut_upper_bound, and never looser than
// the cut so far), then the compaction of the
// CTA's slice: entries with M_hat <= cut are appended to (m_out, i_out) (order not kept:
// the final ordering sorts by (M64, draw index)) and counted straight into the other
// parity's level-0 histogram for the next chunk (the kept entries are few).
__global__ void __launch_bounds__(kSelThreads)
k_sel_keep(const float* __restrict__ ret_m, const uint64_t* __restrict__ ret_i, int64_t nr,
           const float* __restrict__ chunk, int64_t nc, uint64_t first, int new_cut, int par, CutParams cp,
           SelState* __restrict__ st, float* __restrict__ m_out, uint64_t* __restrict__ i_out, int64_t cap_out)
{
    pdl_wait();
    pdl_launch_dependents();
    __shared__ float s_cut;
    const int tid = threadIdx.x, lane = tid & 31;
    // every CTA derives the same cut; a CTA that reads the cut after CTA 0 stored the new one
    // gets the same minimum
    float cut = st->cut;
    if (new_cut) {
        unsigned p2;
        long long k2;
        find_bin(st->hist1[par], st->krem, &p2, &k2);
        if (tid == 0) {
            const uint32_t up_bits = (st->p1 << 20) | (p2 << 8) | 0xFFu;
            s_cut = fminf(cut_upper_bound(cp, __uint_as_float(up_bits)), cut);
        }
        __syncthreads();
        cut = s_cut;
        if (blockIdx.x == 0 && tid == 0) st->cut = cut;
    }
    unsigned* h_next = st->hist0[1 - par];
    const int64_t N = nr + nc, per = sel_slice(N, gridDim.x);
    const int64_t lo = std::min<int64_t>(N, (int64_t)blockIdx.x * per), hi = std::min<int64_t>(N, lo + per);
    for (int64_t base = lo; base < hi; base += (int64_t)kSelThreads * kSelUnroll) {
        float v[kSelUnroll];
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const int64_t e = base + (int64_t)u * kSelThreads + tid;
            v[u] = e < hi ? sel_elem(ret_m, nr, chunk, e) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSelUnroll; ++u) {
            const int64_t e = base + (int64_t)u * kSelThreads + tid;
            const bool keep = e < hi && v[u] <= cut;
            warp_count(h_next, keep, __float_as_uint(v[u]) >> 20);
            const unsigned m = __ballot_sync(kFull, keep);
            if (m == 0) continue;
            unsigned long long pos0 = 0;
            if (lane == 0) pos0 = atomicAdd(reinterpret_cast<unsigned long long*>(&st->kept), (unsigned long long)__popc(m));
            pos0 = __shfl_sync(kFull, pos0, 0);
            if (keep) {
                const unsigned long long pos = pos0 + (unsigned long long)__popc(m & ((1u << lane) - 1u));
                if (pos < (unsigned long long)cap_out) {
                    m_out[pos] = v[u];
                    i_out[pos] = e < nr ? ret_i[e] : first + (uint64_t)(e - nr);
                }
            }
        }
    }
}

// State of a new stream: both histogram sets cleared, the cut, the counters and the
// end-of-stream fields (boundary M64 = NaN until the finish finds them).
__global__ void __launch_bounds__(kSelThreads) k_sel_init(SelState* __restrict__ st, float cut)
{
    unsigned* h = &st->hist0[0][0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * kBins; i += gridDim.x * blockDim.x) h[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->p1 = 0;
        st->krem = 0;
        st->cut = cut;
        st->kept = 0;
        st->nsel = 0;
        st->boundary[0] = st->boundary[1] = __longlong_as_double(0x7FF8000000000000ll);
        st->max_rel = st->max_over_band = st->thr = 0.0;
        st->violations = 0;
        st->err = 0;
        st->fin_overflow = 0;
    }
}

// ------------------------------------------------------------- one-CTA finish --
// The exact M of every retained draw is known (the recheck); what is left is the order.
// One CTA of 1024 threads holds the r <= kFinMax retained pairs (M64, draw index), one to
// four per thread. M64 >= 0 orders like its bit pattern, so in q mode the K-th smallest M64
// is found by a radix select on the 64-bit patterns (8 bits per pass, from the first bit in
// which the smallest and largest pattern differ); an entry is accepted when its M64 is
// smaller, or equal and among the first (K minus the smaller ones) of the equal entries in
// draw order. Threshold mode accepts M64 <= a. Each accepted entry is then placed at the
// number of accepted entries with a smaller draw index (one warp per entry), and one thread
// writes the summary the host reads back.
constexpr int kFinMax = 4096;
constexpr int kFinThreads = SNT;
constexpr int kFinPer = kFinMax / kFinThreads;   // entries per thread
constexpr int kFinCountMax = 512;  // above this many accepted entries the placement sorts instead of counting

__global__ void __launch_bounds__(kFinThreads, 1)
k_finish(const double* __restrict__ m64, const uint64_t* __restrict__ idx, const float* __restrict__ mhat, int64_t r_host,
         const long long* __restrict__ r_dev, long long K, int q_mode, long long thr_bits, CutParams cp,
         const int* __restrict__ err_word, SelState* __restrict__ st, uint64_t* __restrict__ keys_out,
         double* __restrict__ m_out)
{
    pdl_wait();
    pdl_launch_dependents();
    extern __shared__ unsigned long long fin_smem[];
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_red[32][2];
    __shared__ float s_rel[32], s_band[32];
    __shared__ int s_viol[32];
    __shared__ unsigned long long s_prefix;
    __shared__ long long s_k, s_ntie;
    __shared__ unsigned s_cnt;                  // entries in the bin of rank k after a pass
    __shared__ unsigned long long s_small[32];  // those entries, when there are at most 32
    __shared__ int s_nsmall;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a device count above the bound belongs to an overflowed buffer: the host redoes the selection
    const int64_t r = r_dev ? (*r_dev < r_host ? *r_dev : r_host) : r_host;
    if (r > kFinMax) {
        if (tid == 0) {
            st->fin_overflow = 1;
            st->nsel = 0;
            st->err = *err_word;
        }
        return;
    }
    if (r <= 0) {
        if (tid == 0) {
            const double nan = __longlong_as_double(0x7FF8000000000000ll);
            st->nsel = 0;
            st->boundary[0] = st->boundary[1] = nan;
            st->thr = -INFINITY;
            st->max_rel = st->max_over_band = 0.0;
            st->violations = 0;
            st->fin_overflow = 0;
            st->err = *err_word;
        }
        return;
    }
    unsigned long long* sk = fin_smem;             // M64 bit patterns
    unsigned long long* si = fin_smem + kFinMax;   // draw indices
    int* sflag = reinterpret_cast<int*>(fin_smem + 2 * kFinMax);  // accepted (1) or not (0)
    unsigned long long key[kFinPer];
    unsigned long long lo_key = ~0ull, hi_key = 0ull;
    float mrel = 0.f, mband = 0.f;
    int viol = 0;
#pragma unroll
    for (int m = 0; m < kFinPer; ++m) {
        if (m * kFinThreads >= r) break;  // the same for the whole block
        const int c = tid + m * kFinThreads;
        key[m] = ~0ull;
        if (c < r) {
            const double mv = m64[c];
            key[m] = (unsigned long long)__double_as_longlong(mv);
            sk[c] = key[m];
            si[c] = idx[c];
            lo_key = key[m] < lo_key ? key[m] : lo_key;
            hi_key = key[m] > hi_key ? key[m] : hi_key;
            // diagnostics only: FP32 is enough (and cheap on B300)
            const float a = mhat[c], mf = (float)mv;
            const float err = fabsf(a - mf);
            const float band =
                (float)cp.safety * ((float)cp.lin * sqrtf(fmaxf(a, 0.f)) + (float)cp.quad + (float)cp.rel * a);
            if (mf > 0.f) mrel = fmaxf(mrel, __fdividef(err, mf));
            if (band > 0.f) mband = fmaxf(mband, __fdividef(err, band));
            viol += (err > band) ? 1 : 0;
        }
    }
    for (int off = 16; off >= 1; off >>= 1) {
        mrel = fmaxf(mrel, __shfl_xor_sync(kFull, mrel, off));
        mband = fmaxf(mband, __shfl_xor_sync(kFull, mband, off));
        viol += __shfl_xor_sync(kFull, viol, off);
        const unsigned long long a = __shfl_xor_sync(kFull, lo_key, off), b = __shfl_xor_sync(kFull, hi_key, off);
        lo_key = a < lo_key ? a : lo_key;
        hi_key = b > hi_key ? b : hi_key;
    }
    if (lane == 0) {
        s_rel[warp] = mrel;
        s_band[warp] = mband;
        s_viol[warp] = viol;
        s_red[warp][0] = lo_key;
        s_red[warp][1] = hi_key;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kFinThreads / 32; ++w) {
            lo_key = s_red[w][0] < lo_key ? s_red[w][0] : lo_key;
            hi_key = s_red[w][1] > hi_key ? s_red[w][1] : hi_key;
        }
        s_red[0][0] = lo_key;
        s_red[0][1] = hi_key;
    }
    __syncthreads();
    lo_key = s_red[0][0];
    hi_key = s_red[0][1];

    // the accepted set: key < thr, plus the first `need` entries equal to thr in draw order
    unsigned long long thr;
    long long need;
    if (q_mode) {
        // radix select of the K-th smallest key (K <= r here), from the first differing bit
        unsigned long long prefix = 0ull;
        long long k = K < r ? K : r;
        const int top = (lo_key == hi_key) ? -1 : 63 - __clzll((long long)(lo_key ^ hi_key));
        prefix = top < 0 ? lo_key : (top >= 63 ? 0ull : (lo_key >> (top + 1)) << (top + 1));
        for (int shift = top - 7; top >= 0; shift -= 8) {
            const int sh = shift < 0 ? 0 : shift;
            const int bits = shift < 0 ? 8 + shift : 8;        // the last pass may take fewer bits
            const unsigned long long himask = (sh + bits >= 64) ? 0ull : (~0ull << (sh + bits));
            if (tid < 256) hist[tid] = 0u;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < kFinPer; ++m) {
                if (m * kFinThreads >= r) break;  // the same for the whole block
                const int c = tid + m * kFinThreads;
                const bool take = c < r && (key[m] & himask) == (prefix & himask);
                const unsigned d = take ? (unsigned)((key[m] >> sh) & ((1u << bits) - 1u)) : 0u;
                const unsigned peers = __match_any_sync(kFull, take ? d : 0xffffffffu);
                if (take && (__ffs(peers) - 1) == lane) atomicAdd(&hist[d], (unsigned)__popc(peers));
            }
            __syncthreads();
            if (warp == 0) {
                // digit holding rank k: lane l scans bins 8l .. 8l + 7
                unsigned cnt[8];
                long long mine = 0;
#pragma unroll
                for (int i = 0; i < 8; ++i) { cnt[i] = hist[8 * lane + i]; mine += cnt[i]; }
                long long incl = mine;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const long long y = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off) incl += y;
                }
                long long run = incl - mine;
                if (run < k && k <= incl) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (run < k && k <= run + (long long)cnt[i]) {
                            s_prefix = (prefix & himask) | ((unsigned long long)(8 * lane + i) << sh);
                            s_k = k - run;
                            s_cnt = cnt[i];
                        }
                        run += cnt[i];
                    }
                }
            }
            __syncthreads();
            prefix = s_prefix;
            k = s_k;
            if (shift <= 0) break;
            if (s_cnt <= 32) {
                // At most 32 entries share the prefix so far: gather them and let one warp find
                // the k-th smallest of them (each lane counts the keys below and up to its own),
                // instead of further passes over the remaining low bits.
                const unsigned long long lmask = ~0ull << sh;
                if (tid == 0) s_nsmall = 0;
                __syncthreads();
#pragma unroll
                for (int m = 0; m < kFinPer; ++m) {
                    if (m * kFinThreads >= r) break;  // the same for the whole block
                    const int c = tid + m * kFinThreads;
                    if (c < r && (key[m] & lmask) == (prefix & lmask)) s_small[atomicAdd(&s_nsmall, 1)] = key[m];
                }
                __syncthreads();
                if (warp == 0) {
                    const int nb = s_nsmall;
                    const unsigned long long v = lane < nb ? s_small[lane] : ~0ull;
                    int lt = 0, le = 0;
                    for (int j = 0; j < nb; ++j) {
                        const unsigned long long u = s_small[j];
                        lt += u < v ? 1 : 0;
                        le += u <= v ? 1 : 0;
                    }
                    if (lane < nb && lt < k && k <= le) {  // (lanes holding equal keys write the same)
                        s_prefix = v;
                        s_k = k - lt;
                    }
                }
                __syncthreads();
                prefix = s_prefix;
                k = s_k;
                break;
            }
        }
        thr = prefix;  // the K-th smallest key; k of the entries equal to it are accepted
        need = k;
    } else {
        thr = thr_bits < 0 ? 0ull : (unsigned long long)thr_bits;
        need = thr_bits < 0 ? 0 : (long long)kFinMax;  // threshold mode keeps every equal entry
    }
    if (tid == 0) s_ntie = 0;
    __syncthreads();
    // flags: below the threshold key, or equal to it (ranked among the equal ones below)
    int below = 0;
#pragma unroll
    for (int m = 0; m < kFinPer; ++m) {
        if (m * kFinThreads >= r) break;  // the same for the whole block
        const int c = tid + m * kFinThreads;
        if (c < r) {
            const bool lt = q_mode ? key[m] < thr : (thr_bits >= 0 && key[m] <= thr);
            sflag[c] = lt ? 1 : 0;
            if (q_mode && key[m] == thr) atomicAdd(reinterpret_cast<unsigned long long*>(&s_ntie), 1ull);
            below += lt ? 1 : 0;
        }
    }
    __syncthreads();
    if (q_mode) {
        // entries equal to thr: accepted when fewer than `need` equal entries have a smaller
        // draw index (one warp per equal entry; equal M64 are rare, e.g. complement pairs)
        for (int c = warp; c < r; c += kFinThreads / 32) {
            if (sk[c] != thr) continue;
            const unsigned long long ic = si[c];
            int before = 0;
            for (int c2 = lane; c2 < r; c2 += 32) before += (sk[c2] == thr && si[c2] < ic) ? 1 : 0;
            before = (int)__reduce_add_sync(kFull, (unsigned)before);
            if (lane == 0 && before < need) sflag[c] = 1;
        }
    }
    // smallest key above the accepted ones (the (K+1)-th M64) and the accepted count
    unsigned long long above = ~0ull;
#pragma unroll
    for (int m = 0; m < kFinPer; ++m) {
        if (m * kFinThreads >= r) break;  // the same for the whole block
        const int c = tid + m * kFinThreads;
        if (c < r && key[m] > thr && key[m] < above) above = key[m];
    }
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long a = __shfl_xor_sync(kFull, above, off);
        above = a < above ? a : above;
        below += __shfl_xor_sync(kFull, below, off);
    }
    __syncthreads();
    if (lane == 0) {
        s_red[warp][0] = above;
        s_red[warp][1] = (unsigned long long)below;
    }
    __syncthreads();
    if (tid == 0) {
        long long nb = 0;
        for (int w = 0; w < kFinThreads / 32; ++w) {
            above = s_red[w][0] < above ? s_red[w][0] : above;
            nb += (long long)s_red[w][1];
        }
        for (int w = 1; w < kFinThreads / 32; ++w) {
            mrel = fmaxf(mrel, s_rel[w]);
            mband = fmaxf(mband, s_band[w]);
            viol += s_viol[w];
        }
        const long long ns = q_mode ? (K < r ? K : r) : nb;
        const double nan = __longlong_as_double(0x7FF8000000000000ll);
        st->boundary[0] = (q_mode && K >= 1 && K - 1 < r) ? __longlong_as_double((long long)thr) : nan;
        // the (K+1)-th M64: another entry equal to thr if there is one, else the next larger key
        st->boundary[1] = (q_mode && K < r) ? __longlong_as_double((long long)(s_ntie > need ? thr : above)) : nan;
        if (q_mode) st->thr = ns > 0 ? __longlong_as_double((long long)thr) : -INFINITY;
        st->nsel = ns;
        st->max_rel = mrel;
        st->max_over_band = mband;
        st->violations = viol;
        st->fin_overflow = 0;
    }
    __syncthreads();
    // the accepted entries, packed (in any order) into the shared arrays ai / ak
    __shared__ int s_na;
    if (tid == 0) s_na = 0;
    __syncthreads();
    unsigned long long* ai = fin_smem + 2 * kFinMax + kFinMax / 2;   // packed accepted draw indices
    unsigned long long* ak = ai + kFinMax;                           // and their M64 bit patterns
    for (int c0 = 0; c0 < r; c0 += kFinThreads) {
        const int c = c0 + tid;
        const bool a = c < r && sflag[c] != 0;
        const unsigned m = __ballot_sync(kFull, a);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_na, __popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (a) {
            const int q = base + __popc(m & ((1u << lane) - 1u));
            ai[q] = si[c];
            ak[q] = sk[c];
        }
    }
    __syncthreads();
    const int na = s_na;
    // Ascending draw order. Few accepted entries: each is placed at the number of accepted
    // entries with a smaller draw index (one warp per entry). Many (the cost of that grows as
    // na^2): a bitonic sort of the distinct accepted indices, their M64 alongside, over the next
    // power of two (padding sorts last), O(na log^2 na) with one block barrier per stage.
    unsigned long long best = 0ull;
    bool any = false;
    if (na <= kFinCountMax) {
        for (int a = warp; a < na; a += kFinThreads / 32) {
            const unsigned long long ic = ai[a];
            int pos = 0;
            for (int b = lane; b < na; b += 32) pos += ai[b] < ic ? 1 : 0;
            pos = (int)__reduce_add_sync(kFull, (unsigned)pos);
            if (lane == 0) {
                keys_out[pos] = ic;
                m_out[pos] = __longlong_as_double((long long)ak[a]);
                if (!q_mode && (!any || ak[a] > best)) { best = ak[a]; any = true; }
            }
        }
    } else {
        int np = 1;
        while (np < na) np <<= 1;
        for (int i = na + tid; i < np; i += kFinThreads) {
            ai[i] = ~0ull;
            ak[i] = 0ull;
        }
        __syncthreads();
        for (int kk = 2; kk <= np; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int i = tid; i < np; i += kFinThreads) {
                    const int ixj = i ^ jj;
                    if (ixj > i) {
                        const unsigned long long x = ai[i], y = ai[ixj];
                        if ((x > y) == ((i & kk) == 0)) {
                            ai[i] = y;
                            ai[ixj] = x;
                            const unsigned long long t = ak[i];
                            ak[i] = ak[ixj];
                            ak[ixj] = t;
                        }
                    }
                }
                __syncthreads();
            }
        for (int a = tid; a < na; a += kFinThreads) {
            keys_out[a] = ai[a];
            m_out[a] = __longlong_as_double((long long)ak[a]);
            if (!q_mode && (!any || ak[a] > best)) { best = ak[a]; any = true; }
        }
    }
    if (!q_mode) {
        // threshold mode: the largest accepted M64
        __shared__ unsigned long long s_best[32];
        __shared__ int s_any[32];
        // every thread placed entries: the warp's largest first
        const unsigned am = __ballot_sync(kFull, any);
        unsigned long long wb = any ? best : 0ull;
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, wb, off);
            wb = o > wb ? o : wb;
        }
        if (lane == 0) { s_best[warp] = wb; s_any[warp] = am != 0u ? 1 : 0; }
        __syncthreads();
        if (tid == 0) {
            bool a = false;
            unsigned long long b = 0ull;
            for (int w = 0; w < kFinThreads / 32; ++w)
                if (s_any[w] && (!a || s_best[w] > b)) { b = s_best[w]; a = true; }
            st->thr = a ? __longlong_as_double((long long)b) : -INFINITY;
        }
    }
    if (tid == 0) st->err = *err_word;
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
// band statistics of the re-checked draws (the SelTail fields), for retained sets larger than
// the one-CTA finish holds.
__global__ void __launch_bounds__(SNT)
k_sel_summary(const double* __restrict__ m64, const int* __restrict__ rank, const float* __restrict__ mhat, int64_t r_host,
              const long long* __restrict__ r_dev, long long K, int q_mode, long long thr_bits, CutParams cp,
              const int* __restrict__ err_word, SelState* __restrict__ st)
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
        st->fin_overflow = 0;
        st->err = *err_word;
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
                          const long long* count_dev, const uint64_t* draws, uint32_t* rows, int* zero, int nzero)
{
    FRR_CUDA_TRY(ctx, launch_pdl(k_bits<KB>, warp_grid(ctx, count), 256, 0, ctx->stream, seed, exact ? 1 : 0, ctx->binom,
                                 (int)ctx->n, (int)ctx->n1, first, count, count_dev, draws, rows, zero, nzero));
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
                       const uint64_t* draws, uint32_t* rows, const long long* count_dev, int* zero, int nzero)
{
    if (count == 0) return FRR_OK;
    switch (ctx->kb) {
        case 1: return launch_bits_kb<1>(ctx, seed, exact, first, count, count_dev, draws, rows, zero, nzero);
        case 2: return launch_bits_kb<2>(ctx, seed, exact, first, count, count_dev, draws, rows, zero, nzero);
        case 4: return launch_bits_kb<4>(ctx, seed, exact, first, count, count_dev, draws, rows, zero, nzero);
        case 8: return launch_bits_kb<8>(ctx, seed, exact, first, count, count_dev, draws, rows, zero, nzero);
        case 16: return launch_bits_kb<16>(ctx, seed, exact, first, count, count_dev, draws, rows, zero, nzero);
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

frr_status balance_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout,
                          unsigned* hist0)
{
    if (ctx->opts.precision == FRR_F32) return balance_f32_launch(ctx, seed, exact, first, B, Mout);
    return balance_tc_launch(ctx, seed, exact, first, B, Mout, hist0);
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
    k_sel_init<<<8, kSelThreads, 0, ctx->stream>>>(static_cast<SelState*>(ctx->sel), st.cut);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.ms_init = ms_init;
    ctx->stats.boundary_gap_rel = NAN;
    return FRR_OK;
}

// Selection step over the approximate M of draws [first, first + bc) held in Mhat (device):
// k_sel_level1 and k_sel_keep form the cut (q mode) and compact the chunk and the retained set.
// hist_done: the balance kernel already added the chunk's level-0 counts.
frr_status stream_select_step(frr_ctx* ctx, uint64_t first, uint64_t bc, const float* Mhat, bool last, bool hist_done)
{
    StreamState& st = ctx->st;
    SelState* sel = static_cast<SelState*>(ctx->sel);
    const CutParams cp = cut_params(ctx);
    FRR_TRY(ensure_host_pinned(ctx, 256));
    const int in = ctx->ret_cur, out = 1 - in;
    const int par = st.parity;
    const int64_t N = st.retained + (int64_t)bc;
    const int new_cut = (st.q_mode && N > st.K) ? 1 : 0;
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
    if (!hist_done && bc > 0) {
        const unsigned g0 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)bc, kSelThreads),
                                                                               4 * ctx->num_sms));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_hist0, g0, kSelThreads, 0, ctx->stream, Mhat, (int64_t)bc,
                                     &sel->hist0[par][0]));
    }
    // one slice of V per CTA, at most one CTA per SM
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, 2 * kSelThreads), ctx->num_sms));
    auto select_launch = [&](int fresh_cut) -> frr_status {
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_level1, grid, kSelThreads, 0, ctx->stream, (const float*)ctx->ret_m[in],
                                     st.retained, Mhat, (int64_t)bc, (long long)st.K, fresh_cut, par, sel));
        FRR_CUDA_TRY(ctx, launch_pdl(k_sel_keep, grid, kSelThreads, 0, ctx->stream, (const float*)ctx->ret_m[in],
                                     (const uint64_t*)ctx->ret_idx[in], st.retained, Mhat, (int64_t)bc, first, fresh_cut,
                                     par, cp, sel, ctx->ret_m[out], ctx->ret_idx[out], cap));
        FRR_CUDA_TRY(ctx, cudaGetLastError());
        return FRR_OK;
    };
    if (defer) {
        FRR_TRY(select_launch(new_cut));
        if (st.timing) record_ev(ctx, 2);
        st.retained = -1;
        st.retained_bound = std::min<int64_t>(N, cap);
        st.parity = 1 - par;
        ctx->ret_cur = out;
        return FRR_OK;
    }
    for (int attempt = 0;; ++attempt) {
        // a repeat keeps the cut the first launch stored, so it keeps the same set (and
        // k_sel_level1 clears the next chunk's counts again before k_sel_keep adds them)
        FRR_TRY(select_launch(attempt == 0 ? new_cut : 0));
        long long* hk = static_cast<long long*>(ctx->host_pinned);
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk, &sel->kept, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk + 1, ctx->dev_counters + 12, sizeof(int), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        if (st.timing) record_ev(ctx, 2);
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
        FRR_TRY(ensure_retained(ctx, out, kept));
        cap = (int64_t)(ctx->ret_bytes_m[out] / sizeof(float));
    }
    st.parity = 1 - par;
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
        if (st.timing) record_ev(ctx, 0);
        // the split-BF16 balance kernel also adds the chunk's level-0 counts of the selection
        SelState* sel = static_cast<SelState*>(ctx->sel);
        const bool fused = ctx->opts.precision == FRR_SPLIT_BF16;
        FRR_TRY(balance_launch(ctx, st.seed, st.exact, first + off, bc, ctx->Mhat,
                               fused ? &sel->hist0[st.parity][0] : nullptr));
        if (st.timing) record_ev(ctx, 1);
        FRR_TRY(stream_select_step(ctx, first + off, bc, ctx->Mhat, st.seen + off + bc == st.total, fused));
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
        if (st.timing) record_ev(ctx, 0);  // no balance here: an empty interval
        if (st.timing) record_ev(ctx, 1);
        FRR_TRY(stream_select_step(ctx, first + off, bc, Mhat + off, st.seen + off + bc == st.total, false));
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
    if (st.timing) record_ev(ctx, 3);
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
        FRR_TRY(recheck_launch(ctx, st.seed, st.exact, ctx->ret_idx[cur], rb, m64, r_dev));
        // threshold mode: M64 <= a compares as bit patterns (M64 >= 0); a < 0 accepts nothing
        long long thr_bits = -1;
        if (!st.q_mode && st.threshold >= 0.0) memcpy(&thr_bits, &st.threshold, sizeof(thr_bits));
        // The ordering: one CTA sorts the retained set in shared memory when it holds at most
        // kFinMax draws -- known on the host, or (deferred count, q mode) expected because it is
        // about K plus the draws inside the band; a larger deferred set sets fin_overflow and the
        // caller redoes the selection with the count read back. Otherwise rank and place with
        // one warp per entry.
        const bool one_cta = dev_count ? (st.q_mode && st.K <= kFinMax / 4)
                                       : (rb <= (st.q_mode ? kFinMax : kFinMax / 4) && st.K <= kFinMax / 4);
        if (one_cta) {
            // M64 patterns, indices, flags, packed accepted indices and patterns (147 KiB)
            const size_t smem = (size_t)kFinMax * (4 * sizeof(unsigned long long) + sizeof(int));
            FRR_CUDA_TRY(ctx, set_smem_limit(k_finish, (int)smem, ctx->device));
            FRR_CUDA_TRY(ctx, launch_pdl(k_finish, 1, kFinThreads, smem, ctx->stream, (const double*)m64,
                                         (const uint64_t*)ctx->ret_idx[cur], (const float*)ctx->ret_m[cur], rb, r_dev,
                                         (long long)st.K, st.q_mode ? 1 : 0, thr_bits, cut_params(ctx),
                                         (const int*)(ctx->dev_counters + 12), sel, place_k, place_m));
        } else {
            FRR_CUDA_TRY(ctx, launch_pdl(k_rank, warp_grid(ctx, rb), 256, 0, ctx->stream, m64, ctx->ret_idx[cur], rb,
                                         r_dev, rank));
            FRR_CUDA_TRY(ctx, launch_pdl(k_place_sel, warp_grid(ctx, rb), 256, 0, ctx->stream, m64, ctx->ret_idx[cur],
                                         rank, rb, r_dev, (long long)st.K, st.q_mode ? 1 : 0, thr_bits, place_k, place_m));
            FRR_CUDA_TRY(ctx, launch_pdl(k_sel_summary, 1, SNT, 0, ctx->stream, m64, rank, ctx->ret_m[cur], rb, r_dev,
                                         (long long)st.K, st.q_mode ? 1 : 0, thr_bits, cut_params(ctx),
                                         (const int*)(ctx->dev_counters + 12), sel));
        }
        FRR_CUDA_TRY(ctx, cudaGetLastError());
        // kept (the retained count) and the SelTail fields (the device error word included), in one copy
        FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hp, &sel->kept, sizeof(long long) + sizeof(SelTail), cudaMemcpyDeviceToHost,
                                          ctx->stream));
        if (stage) {
            if (host_keys)
                FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hk, kout, (size_t)stage_n * 8, cudaMemcpyDeviceToHost, ctx->stream));
            if (host_m)
                FRR_CUDA_TRY(ctx, cudaMemcpyAsync(hm, mout, (size_t)stage_n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    if (st.timing) record_ev(ctx, 4);
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
        if (tail.err != 0) {
            FRR_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dev_counters + 12, 0, sizeof(int), ctx->stream));
            FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            st.active = false;
            return FRR_E_TIMEOUT;
        }
        if (r > rb || tail.fin_overflow) {
            // the deferred retained set outgrew its buffer (or the one-CTA finish): nothing
            // written; redo undeferred
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
    // q mode accepts exactly min(K, B) draws; anything else is an internal error
    if (st.q_mode && nsel != std::min<int64_t>(st.K, (int64_t)st.total)) return FRR_E_MISMATCH;

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
    st.parity = 0;
    if (h.retained > 0) {
        // the level-0 counts of the restored retained set (stream_begin cleared both sets)
        SelState* sl = static_cast<SelState*>(ctx->sel);
        const unsigned g0 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h.retained, kSelThreads),
                                                                               4 * ctx->num_sms));
        const cudaError_t e = launch_pdl(k_sel_hist0, g0, kSelThreads, 0, ctx->stream, (const float*)ctx->ret_m[0],
                                         (int64_t)h.retained, &sl->hist0[0][0]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->failed = true;
            st.active = false;
            return FRR_E_CUDA;
        }
    }
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
