// frr_recheck_tc.cu -- exact-sum recheck of candidate draws on the tensor cores.
//
// The accepted set is decided on M computed from exact treated sums S_T,j =
// sum_{i in T} Q_ij of the fixed-point covariates Q = round(Zc 2^qexp) (|Q| <= 2^46).
// Q is written in balanced base-4096 digits, Q = sum_{k<4} q_k 4096^k with q_k in
// [-2048, 2047], each digit plane stored in FP16 (exact). For a 0/1 assignment row w
// (FP16 ones), D_k = sum_i w_i q_k(i) is an integer of magnitude below 2^22, so the
// tensor cores' FP32 accumulation of the digit products is exact, and
// S_T = sum_k D_k 4096^k is rebuilt exactly in int64 (Horner). The epilogue then forms, per column, the exact
// 128-bit integer N_j = S_T n - S_all n1 = n1 n0 Delta_j 2^q_j (an assignment and its
// complement give -N_j when n1 = n0), rounds N_j 2^-q_j once to FP64 and adds its square
// to the CTA's partial sum; M64 = sum / (n n1 n0).
//
// Work items of (128 candidates, 64 columns), 4 accumulators of 64 columns in TMEM each,
// taken by persistent CTAs (one per SM at most).
// Warps 0-15 epilogue (warp w: TMEM lanes 32 (w % 4) .., columns 16 (w / 4) .. of the item,
// so four warps share each row and the integer epilogue runs on 16 warps), warp 16 TMA (4
// digit tiles per K block, stacked into one 256-row B tile), warp 17 MMA (all four planes in
// one N = 256 MMA per K step of 16), warps 18-21 expand the candidates' bit rows (computed
// beforehand) into FP16 0/1 A tiles with integer arithmetic.
// The CTA that finishes the last column chunk of a candidate tile also adds up each
// candidate's partial sums (in column order) into its M64.
#include "frr_internal.cuh"

#include <algorithm>
#include "frr_exact.cuh"
#include "frr_gen.cuh"
#include "frr_tc_ptx.cuh"

namespace frr {
using namespace tc;
using namespace exact;
namespace {

constexpr int kM = 128, kN = 64, kPlanes = kDigitPlanes, kKB = 64;
constexpr int kStB = 4, kStA = 2;
constexpr int kPlaneBytes = kN * kKB * 2;          // 8 KiB
constexpr int kBBytes = kPlanes * kPlaneBytes;     // 32 KiB
constexpr int kABytes = kM * kKB * 2;              // 16 KiB
constexpr int kEpiWarps = 16;  // four per TMEM lane quarter, one per 16-column quarter of an item
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kQuarters = 4;   // column quarters of an item (one epilogue thread each per candidate)
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1, kExpWarp0 = kEpiWarps + 2;
constexpr int kThreads = (kExpWarp0 + 4) * 32;
static_assert(kN == 64 && kPlanes * kN == 256, "16-column epilogue quarters; the four planes in one N = 256 MMA");

// Eight FP16 values 0.0 / 1.0 from the bits of byte x (bit i -> element i): y * 0x8001 puts
// bits 0 and 1 of y at positions 0 and 16, and times 0x3C00 (FP16 1.0) makes them halves.
__device__ __forceinline__ uint4 expand_byte_f16(uint32_t x)
{
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = (((x >> (2 * q)) * 0x8001u) & 0x00010001u) * 0x3C00u;
    return make_uint4(w[0], w[1], w[2], w[3]);
}

size_t rc_smem_bytes() { return 1024 + (size_t)kStB * kBBytes + (size_t)kStA * kABytes + 16 * 8 + 16; }

// Persistent: CTA b takes work items b, b + gridDim.x, ... of (column chunk, candidate
// tile), item i -> chunk i / T, tile i % T with T = ceil(C / 128) tiles (consecutive items
// share a chunk's digit tiles in L2). C is read from C_dev when given (a count the host
// has not read back), else C_host.
__global__ void __launch_bounds__(kThreads, 1)
k_recheck_tc(const __grid_constant__ CUtensorMap map_q, const uint32_t* __restrict__ rows, int W, int64_t C_host,
             const long long* __restrict__ C_dev, int nkb, int d, int n, int n1, const long long* __restrict__ Qsum,
             const int* __restrict__ qexp, double* __restrict__ part, int ncb, int* __restrict__ tile_done,
             double denom, double* __restrict__ M64, int* err)
{
    pdl_wait();
    pdl_launch_dependents();
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sB = smem;
    unsigned char* sA = sB + kStB * kBBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sA + kStA * kABytes);
    uint64_t* b_full = bar;
    uint64_t* b_empty = b_full + kStB;
    uint64_t* a_full = b_empty + kStB;
    uint64_t* a_empty = a_full + kStA;
    uint64_t* acc_full = a_empty + kStA;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);
    __shared__ long long sQsum[kN];
    __shared__ int sQexp[kN];
    __shared__ int sLast;   // this CTA completed the last column chunk of the item's candidate tile
    __shared__ double sSum[kQuarters - 1][kM];  // quarter sums: of an item's columns, then of a row's partial sums

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t C = C_dev ? std::min<int64_t>((int64_t)*C_dev, C_host) : C_host;  // within the buffers
    const int64_t T = (C + kM - 1) / kM;
    const int64_t items = T * ncb;
    if (tid == 0) {
        for (int s = 0; s < kStB; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
        for (int s = 0; s < kStA; ++s) { mbar_init(&a_full[s], 4); mbar_init(&a_empty[s], 1); }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kEpiWarps);
        mbar_init(mma_done, 1);
        *sAbort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        tmem_alloc(sTmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *sTmem;

    if (warp == kTmaWarp) {
        if (lane == 0) {
            uint32_t bi = 0;
            bool ok = true;
            for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
                const int chunk = (int)(item / T);
                for (int kb = 0; kb < nkb; ++kb, ++bi) {
                    const int s = bi % kStB;
                    if (!(ok = wait_bar(&b_empty[s], ((bi / kStB) & 1u) ^ 1u, sAbort, err, 11))) break;
                    mbar_arrive_expect_tx(&b_full[s], kBBytes);
                    for (int pl = 0; pl < kPlanes; ++pl)
                        tma_load_2d(sB + s * kBBytes + pl * kPlaneBytes, &map_q, &b_full[s], kb * kKB,
                                    pl * d + chunk * kN);
                }
            }
            if (!ok) {
                // drain the copies this thread may still have in flight
                const uint32_t from = bi > (uint32_t)kStB ? bi - kStB : 0u;
                for (uint32_t i = from; i < bi; ++i) {
                    const unsigned long long t0 = clock64();
                    while (!mbar_try_wait(&b_full[i % kStB], (i / kStB) & 1u) && clock64() - t0 < kWaitCycles) {}
                }
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            bool ok = true;
            uint32_t ai = 0, bi = 0, it = 0;
            // the four planes (rows 0-255 of the stacked B tile) in one N = 256 MMA: the 0/1 A
            // tile is read once per K step
            const uint32_t idesc4 = idesc_f16(kM, kPlanes * kN);
            for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
                if (!(ok = wait_bar(acc_empty, (it & 1u) ^ 1u, sAbort, err, 16))) break;
                tc_fence_after();
                for (int kb = 0; kb < nkb && ok; ++kb, ++ai, ++bi) {
                    const int sa = ai % kStA, sb = bi % kStB;
                    if (!(ok = wait_bar(&a_full[sa], (ai / kStA) & 1u, sAbort, err, 12))) break;
                    if (!(ok = wait_bar(&b_full[sb], (bi / kStB) & 1u, sAbort, err, 13))) break;
                    tc_fence_after();
                    const uint64_t adesc = sdesc_sw128(smem_u32(sA + sa * kABytes));
                    const uint64_t bdesc4 = sdesc_sw128(smem_u32(sB + sb * kBBytes));
#pragma unroll
                    for (int k = 0; k < kKB / 16; ++k)
                        umma_bf16(tmem_base, adesc + 2u * k, bdesc4 + 2u * k, idesc4, (kb | k) != 0 ? 1u : 0u);
                    umma_commit(&b_empty[sb]);
                    umma_commit(&a_empty[sa]);
                }
                if (ok) umma_commit(acc_full);
            }
            // every MMA this thread issued has finished before TMEM is released
            umma_commit(mma_done);
            const unsigned long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {}
        }
    } else if (warp >= kExpWarp0) {
        const int r = tid - kExpWarp0 * 32;  // row (candidate) of the A tile
        uint32_t ai = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const int64_t cand = (item % T) * kM + r;
            const uint32_t* rw = rows + (cand < C ? cand : 0) * (int64_t)W;
            // the row words of the next K block are loaded while this one is expanded
            uint2 nxt = make_uint2(0u, 0u);
            if (cand < C && nkb > 0) nxt = *reinterpret_cast<const uint2*>(rw);
            for (int kb = 0; kb < nkb && ok; ++kb, ++ai) {
                const int s = ai % kStA;
                const uint32_t w2[2] = {nxt.x, nxt.y};
                if (cand < C && kb + 1 < nkb) nxt = *reinterpret_cast<const uint2*>(rw + 2 * (kb + 1));
                if (!(ok = wait_bar(&a_empty[s], ((ai / kStA) & 1u) ^ 1u, sAbort, err, 14))) break;
                unsigned char* dst = sA + s * kABytes + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t x = (w2[q >> 2] >> (8 * (q & 3))) & 0xFFu;
                    *reinterpret_cast<uint4*>(dst + ((q ^ (r & 7)) << 4)) = expand_byte_f16(x);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[s]);
            }
        }
    } else {
        // epilogue: candidate row 32 (warp % 4) + lane, column quarter warp / 4 of the item
        const int row = 32 * (warp & 3) + lane, qtr = warp >> 2;
        uint32_t it = 0;
        bool ok = true;
        for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x, ++it) {
            const int chunk = (int)(item / T);
            const int64_t cand = (item % T) * kM + row;
            // the chunk's column sums and scales (the previous item's readers are done first)
            asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
            for (int t = tid; t < kN; t += 32 * kEpiWarps) {
                const int col = chunk * kN + t;
                sQsum[t] = col < d ? Qsum[col] : 0ll;
                sQexp[t] = col < d ? qexp[col] : 0;
            }
            asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
            if (!(ok = wait_bar(acc_full, it & 1u, sAbort, err, 15))) break;
            tc_fence_after();
            double psum = 0.0;
            const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16);
            // n1 n0 Delta_j 2^q_j = S_T n0 - S_C n1 = S_T n - S_all n1 =: N_j, an exact 128-bit
            // integer; when n1 = n0 the complement (S_T -> S_all - S_T) gives exactly -N_j.
            // N_j 2^-q_j is rounded once to FP64 with integer instructions and squared into
            // the partial sum: one FP64 operation per column (B300's FP64 unit is narrow).
            {
                const int c0 = 16 * qtr;
                long long S[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) S[j] = 0;
                for (int pl = kPlanes - 1; pl >= 0; --pl) {
                    uint32_t v[16];
                    tmem_ld16(taddr + (uint32_t)(pl * kN + c0), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        S[j] = S[j] * (1ll << kDigitBits) + (long long)acc_to_int(__uint_as_float(v[j]));
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = chunk * kN + c0 + j;
                    if (col < d) {
                        const long long Q = sQsum[c0 + j];
                        const unsigned long long a_lo = (unsigned long long)S[j] * (unsigned long long)n;
                        const long long a_hi = __mul64hi(S[j], (long long)n);
                        const unsigned long long b_lo = (unsigned long long)Q * (unsigned long long)n1;
                        const long long b_hi = __mul64hi(Q, (long long)n1);
                        const unsigned long long lo = a_lo - b_lo;
                        const long long hi = a_hi - b_hi - (a_lo < b_lo ? 1ll : 0ll);
                        const double x = i128_to_double_scaled(hi, lo, sQexp[c0 + j]);
                        psum = __fma_rn(x, x, psum);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
            // the four quarter sums of the item, added in column order inside this CTA: one
            // partial sum per (candidate, column chunk), so the tile's last CTA adds ncb of them
            // per candidate rather than 4 ncb (the FP64 unit is narrow)
            if (qtr > 0) sSum[qtr - 1][row] = psum;
            asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
            if (qtr == 0 && cand < C) {
#pragma unroll
                for (int q = 0; q < kQuarters - 1; ++q) psum = __dadd_rn(psum, sSum[q][row]);
                part[cand * ncb + chunk] = psum;
            }
            // The CTA that completes the last of a tile's ncb column chunks sums each candidate's
            // ncb partial sums in column order and forms M64 = sum / (n n1 n0). Thread 0 counts
            // for the CTA: a fence before the count publishes the CTA's partial sums (written
            // before the barrier), and in the last CTA a fence after it orders the other CTAs'
            // partial sums before the loads that follow the second barrier.
            asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
            if (tid == 0) {
                __threadfence();
                sLast = atomicAdd(&tile_done[item % T], 1) == ncb - 1;
                if (sLast) __threadfence();
            }
            asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
            if (sLast) {
                // thread (row, quarter qtr) adds the row's partial sums [lo, hi) -- a quarter of its
                // ncb, one per column chunk -- in column order, sixteen loads in flight; the
                // quarters are then added in order, and M64 = sum / (n n1 n0)
                const int per = (ncb + kQuarters - 1) / kQuarters;
                const int lo = qtr * per, hi = lo + per < ncb ? lo + per : ncb;
                const double* pc = part + cand * (int64_t)ncb;
                double s = 0.0;
                if (cand < C) {
                    for (int b0 = lo; b0 < hi; b0 += 16) {
                        double v[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) v[u] = b0 + u < hi ? __ldcg(pc + b0 + u) : 0.0;
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (b0 + u < hi) s = __dadd_rn(s, v[u]);
                    }
                }
                if (qtr > 0) sSum[qtr - 1][row] = s;
                asm volatile("bar.sync 1, %0;" :: "n"(kEpiThreads) : "memory");
                if (qtr == 0 && cand < C) {
#pragma unroll
                    for (int q = 0; q < kQuarters - 1; ++q) s = __dadd_rn(s, sSum[q][row]);
                    M64[cand] = __ddiv_rn(__dmul_rn(1.0, s), denom);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

}  // namespace

// Exact-sum recheck of `count` draws (device list) on the tensor cores; M64 on the device.
// With count_dev the number of draws is read on the device and `count` only bounds it.
frr_status recheck_tc_launch(frr_ctx* ctx, uint64_t seed, bool exact, const uint64_t* draws, int64_t count,
                             double* M64, const long long* count_dev)
{
    if (count <= 0) return FRR_OK;
    const int W = 4 * ctx->kb;
    const int ncb = ceil_div(ctx->d, kN);
    const int64_t tiles = (count + kM - 1) / kM;
    const size_t rows_bytes = ((size_t)count * W * sizeof(uint32_t) + 255) & ~size_t(255);
    const size_t part_bytes = ((size_t)count * ncb * sizeof(double) + 255) & ~size_t(255);
    const size_t ctr_bytes = (size_t)tiles * sizeof(int);
    FRR_TRY(ensure_device(ctx, &ctx->misc2, &ctx->misc2_bytes, rows_bytes + part_bytes + ctr_bytes));
    uint32_t* rows = static_cast<uint32_t*>(ctx->misc2);
    double* part = reinterpret_cast<double*>(static_cast<char*>(ctx->misc2) + rows_bytes);
    int* tile_done = reinterpret_cast<int*>(static_cast<char*>(ctx->misc2) + rows_bytes + part_bytes);
    // the bit rows, and the per-tile completion counters zeroed before the recheck counts on them
    FRR_TRY(bits_launch(ctx, seed, exact, 0, (uint64_t)count, draws, rows, count_dev, tile_done, (int)tiles));
    if (!ctx->qmap_ready) {
        if (!make_map_f16(&ctx->qmap, ctx->Zq, (uint64_t)ctx->kpad, (uint64_t)kPlanes * ctx->d, kKB, kN))
            return FRR_E_CUDA;
        ctx->qmap_ready = true;
    }
    const size_t smem = rc_smem_bytes();
    FRR_CUDA_TRY(ctx, set_smem_limit(k_recheck_tc, (int)smem, ctx->device));
    const int64_t items = (int64_t)((count + kM - 1) / kM) * ncb;
    const unsigned grid = (unsigned)std::min<int64_t>(items, ctx->num_sms);
    // the partial sums hold (N_j 2^-q_j)^2 = (n1 n0 Delta_j)^2, and M = (n1 n0 / n) sum Delta_j^2
    const double denom = (double)ctx->n * (double)ctx->n1 * (double)ctx->n0;
    FRR_CUDA_TRY(ctx, launch_pdl(k_recheck_tc, grid, kThreads, smem, ctx->stream, ctx->qmap, rows, W, count, count_dev,
                                 ctx->kused / kKB, (int)ctx->d, (int)ctx->n, (int)ctx->n1, ctx->Qsum, ctx->qexp, part,
                                 ncb, tile_done, denom, M64, ctx->dev_counters + 12));
    return FRR_OK;
}

}  // namespace frr
