// frr_balance_tc.cu -- split-BF16 tensor-core balance check (tcgen05 + TMA + TMEM), sm_103a.
//
// Hotelling T^2 of each draw (Sec. 2.2, 2.3): s_b = w_b^T Zc, M_b = n/(n1 n0) ||s_b||^2.
// W is 0/1, exact in BF16; Zc is split into BF16 parts hi = bf16(Zc), lo = bf16(Zc - hi),
// and both products accumulate into one FP32 accumulator: s = W.hi + W.lo.
//
// One persistent CTA per SM walks tiles of up to 128 consecutive draws (a single experiment:
// a contiguous range of ceil(B / CTAs) draws per CTA with the remainder in its first tile; a
// batch: the table's tiles dealt round-robin). Warp roles:
//   warps 0-3   epilogue: tcgen05.ld of the accumulator (TMEM lane = draw), sum of
//               squares over the covariate chunks, M_hat written per draw;
//   warp 4      TMA producer: Zc hi / lo tiles (256 covariates x 64 K positions, 128B
//               swizzle) into a 4-stage shared-memory ring;
//   warp 5      TMEM allocator and MMA issuer (one thread): per covariate chunk of
//               N <= 256 columns, 2 x 4 tcgen05.mma (M=128, K=16) per 64-wide K block
//               into one of two TMEM accumulators (2 x 256 columns);
//   warps 6-9   A producer: expand the draws' bit rows into BF16 0/1 K-major tiles
//               (128 x 64, 128B swizzle), one draw row per thread, through a 256-entry
//               byte table in shared memory;
//   warps 10..  generation (NG warps): Philox + warp select (frr_gen.cuh) of the
//               next tile's 128 draws into a double-buffered bit-row buffer.
// The assignment matrix exists only as bits and BF16 tiles in shared memory.
// Every mbarrier wait is bounded (about one second); on expiry the CTA records an
// error word, drains its own TMA copies, frees TMEM and returns.
#include "frr_internal.cuh"
#include "frr_gen.cuh"

#include <cuda.h>

#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "frr_tcexp.cuh"
#include "frr_tc_ptx.cuh"

namespace frr {
using namespace tc;
namespace {

constexpr int kTileM = 128;          // draws per tile = TMEM lanes
constexpr int kChunkN = 256;         // covariates per accumulator chunk
constexpr int kKBlock = 64;          // K positions per stage (128 bytes of BF16)
constexpr int kStagesA = 3;
constexpr int kBBytes = kChunkN * kKBlock * 2;   // 32 KiB
constexpr int kABytes = kTileM * kKBlock * 2;    // 16 KiB
constexpr int kExpWarps = 4;   // 128 threads: one A-tile row each

}  // namespace

namespace {


// Experiment and local tile index of global tile g: the single experiment `one`, or
// the entry e of `table` with prefix[e] <= g < prefix[e + 1].
__device__ __forceinline__ const TcExp* tile_job(const TcExp* one, const TcExp* table, const unsigned long long* prefix,
                                                 int E, uint64_t g, uint64_t& tl)
{
    if (table == nullptr) { tl = g; return one; }
    int lo = 0, hi = E;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid;
    }
    tl = g - prefix[lo];
    return table + lo;
}

// The tiles of one CTA. Batched launch: global tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// of the table. Single experiment: the CTA owns a contiguous range of D = ceil(B / gridDim.x)
// draws cut into tiles of 128 with the remainder first, so that the first tile -- whose bit
// rows must all be generated before the CTA's first MMA -- is the smallest, and every CTA
// runs the same number of tiles (a draw's M_hat does not depend on the tile it is in).
struct TileSched {
    uint64_t lo;         // single experiment: the CTA's first draw
    uint64_t count;      // tiles of this CTA
    int first;           // single experiment: draws in the first tile
};

__device__ __forceinline__ TileSched tile_sched(const TcExp& one, const TcExp* table, unsigned long long tiles)
{
    TileSched s{0, 0, 0};
    if (table != nullptr) {
        s.count = blockIdx.x < tiles ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
        return s;
    }
    const uint64_t D = (one.B + gridDim.x - 1) / gridDim.x;
    s.lo = (uint64_t)blockIdx.x * D;
    const uint64_t n = s.lo < one.B ? (one.B - s.lo < D ? one.B - s.lo : D) : 0;
    s.count = (n + kTileM - 1) / kTileM;
    s.first = s.count ? (int)(n - (s.count - 1) * kTileM) : 0;
    return s;
}

// Tile i of the CTA: its experiment, first draw offset (relative to the experiment's first
// draw) and number of draws (<= 128).
__device__ __forceinline__ const TcExp* tile_at(const TileSched& sc, const TcExp* one, const TcExp* table,
                                                const unsigned long long* prefix, int E, uint64_t i, uint64_t& base,
                                                int& cnt)
{
    if (table == nullptr) {
        base = sc.lo + (i == 0 ? 0 : (uint64_t)sc.first + (i - 1) * kTileM);
        cnt = i == 0 ? sc.first : kTileM;
        return one;
    }
    uint64_t tl;
    const TcExp* x = tile_job(one, table, prefix, E, blockIdx.x + i * gridDim.x, tl);
    base = tl * kTileM;
    cnt = x->B - base < (uint64_t)kTileM ? (int)(x->B - base) : kTileM;
    return x;
}

// Bit row of one draw for a run-time number of Philox blocks per lane kb <= KBMAX.
template <int KBMAX>
__device__ __forceinline__ void draw_bits_kb(int kb, bool exact, uint64_t seed, uint64_t draw, int n, int n1,
                                             const uint64_t* binom, uint32_t* row, int lane)
{
    if constexpr (KBMAX >= 16) { if (kb == 16) { warp_draw_bits<16>(exact, seed, draw, n, n1, binom, row, lane); return; } }
    if constexpr (KBMAX >= 8) { if (kb == 8) { warp_draw_bits<8>(exact, seed, draw, n, n1, binom, row, lane); return; } }
    if constexpr (KBMAX >= 4) { if (kb == 4) { warp_draw_bits<4>(exact, seed, draw, n, n1, binom, row, lane); return; } }
    if constexpr (KBMAX >= 2) { if (kb == 2) { warp_draw_bits<2>(exact, seed, draw, n, n1, binom, row, lane); return; } }
    warp_draw_bits<1>(exact, seed, draw, n, n1, binom, row, lane);
}

template <int KB, int SB, int NG, bool MULTI>
__global__ void __launch_bounds__((6 + kExpWarps + NG) * 32, 1)
k_balance_tc(const __grid_constant__ TcExp one, const TcExp* __restrict__ table,
             const unsigned long long* __restrict__ prefix, int E, unsigned long long tiles, int* err)
{
    constexpr int W = 4 * KB;  // bit-row words per draw
    constexpr int RS = W + 1;  // odd row stride: the expansion threads read 32 rows without bank conflicts
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sB = smem;                                    // SB x 32 KiB
    unsigned char* sA = sB + SB * kBBytes;                       // kStagesA x 16 KiB
    uint32_t* sBits = reinterpret_cast<uint32_t*>(sA + kStagesA * kABytes);  // 2 x 128 x RS
    uint64_t* bar = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(sBits + 2 * kTileM * RS) + 7) & ~uintptr_t(7));
    uint64_t* b_full = bar;
    uint64_t* b_empty = b_full + SB;
    uint64_t* a_full = b_empty + SB;
    uint64_t* a_empty = a_full + kStagesA;
    uint64_t* acc_full = a_empty + kStagesA;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* bits_full = acc_empty + 2;
    uint64_t* bits_empty = bits_full + 2;
    uint64_t* mma_done = bits_empty + 2;
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ uint4 sLut8[256];   // byte -> eight BF16 values 0.0 / 1.0 (bit i -> value i)
    if (tid < 256) {
        uint32_t h[8];
        for (int i = 0; i < 8; ++i) h[i] = ((tid >> i) & 1) ? 0x3F80u : 0u;
        sLut8[tid] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
    }

    if (tid == 0) {
        for (int s = 0; s < SB; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
        for (int s = 0; s < kStagesA; ++s) { mbar_init(&a_full[s], kExpWarps); mbar_init(&a_empty[s], 1); }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
            mbar_init(&bits_full[s], NG);
            mbar_init(&bits_empty[s], kExpWarps);
        }
        mbar_init(mma_done, 1);
        *sAbort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        tmem_alloc(sTmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *sTmem;
    const TileSched sched = tile_sched(one, table, tiles);
    // limit of every bounded wait (shortened only by the failure-path test, see frr_test_wait_expiry)
    const unsigned long long wlim = one.wait_cycles ? one.wait_cycles : kWaitCycles;

    if (warp == 4) {
        // ------------------------------------------------------------ TMA --
        if (lane == 0 && !one.skip_tma) {
            uint32_t bi = 0;
            bool ok = true;
            for (uint64_t i = 0; i < sched.count && ok; ++i) {
                uint64_t base;
                int cnt;
                const TcExp* x = tile_at(sched, &one, table, prefix, E, i, base, cnt);
                const int nch = x->nchunks, nkb = x->nkb;
                for (int c = 0; c < nch && ok; ++c)
                    for (int kb = 0; kb < nkb && ok; ++kb)
                        for (int part = 0; part < 2 && ok; ++part, ++bi) {
                            const int s = bi % SB;
                            const uint32_t ph = (bi / SB) & 1u;
                            if (!(ok = wait_bar(&b_empty[s], ph ^ 1u, sAbort, err, 1, wlim))) break;
                            mbar_arrive_expect_tx(&b_full[s], kBBytes);
                            tma_load_2d(sB + s * kBBytes, part ? &x->map_lo : &x->map_hi, &b_full[s], kb * kKBlock,
                                        c * kChunkN);
                        }
            }
            if (!ok) {
                // drain the copies this thread may still have in flight
                const uint32_t from = bi > (uint32_t)SB ? bi - SB : 0u;
                for (uint32_t i = from; i < bi; ++i) {
                    const unsigned long long t0 = clock64();
                    while (!mbar_try_wait(&b_full[i % SB], (i / SB) & 1u) && clock64() - t0 < kWaitCycles) {}
                }
            }
        }
    } else if (warp == 5) {
        // ------------------------------------------------------------ MMA --
        if (lane == 0) {
            uint32_t ai = 0, bi = 0, g = 0;
            bool ok = true;
            for (uint64_t i = 0; i < sched.count && ok; ++i) {
                uint64_t base;
                int cnt;
                const TcExp* x = tile_at(sched, &one, table, prefix, E, i, base, cnt);
                const int nch = x->nchunks, nkb = x->nkb, dd = x->d;
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int buf = g & 1;
                    if (!(ok = wait_bar(&acc_empty[buf], ((g >> 1) & 1u) ^ 1u, sAbort, err, 2, wlim))) break;
                    tc_fence_after();
                    const int rem = dd - c * kChunkN;
                    const int N = rem >= kChunkN ? kChunkN : ((rem + 15) / 16) * 16;
                    const uint32_t idesc = idesc_bf16(kTileM, N);
                    const uint32_t dt = tmem_base + (uint32_t)(buf * kChunkN);
                    for (int kb = 0; kb < nkb && ok; ++kb, ++ai) {
                        const int sa = ai % kStagesA;
                        if (!(ok = wait_bar(&a_full[sa], (ai / kStagesA) & 1u, sAbort, err, 3, wlim))) break;
                        const uint64_t adesc = sdesc_sw128(smem_u32(sA + sa * kABytes));
                        for (int part = 0; part < 2; ++part, ++bi) {
                            const int sb = bi % SB;
                            if (!(ok = wait_bar(&b_full[sb], (bi / SB) & 1u, sAbort, err, 4, wlim))) break;
                            tc_fence_after();
                            const uint64_t bdesc = sdesc_sw128(smem_u32(sB + sb * kBBytes));
#pragma unroll
                            for (int k = 0; k < kKBlock / 16; ++k)
                                umma_bf16(dt, adesc + 2u * k, bdesc + 2u * k, idesc, (kb | part | k) != 0 ? 1u : 0u);
                            umma_commit(&b_empty[sb]);
                        }
                        if (ok) umma_commit(&a_empty[sa]);
                    }
                    if (ok) umma_commit(&acc_full[buf]);
                }
            }
            // every MMA this thread issued has finished before TMEM is released
            umma_commit(mma_done);
            const unsigned long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {}
        }
    } else if (warp >= 6 && warp < 6 + kExpWarps) {
        // ------------------------------------------------- A tile producer --
        // thread r writes row r (draw r of the tile): the 64 bits of K block kb become
        // eight 16-byte chunks of BF16 0.0 / 1.0 (one byte-table entry each), chunk q
        // stored at (q ^ (r % 8)).
        const int r = tid - 6 * 32;  // 0..127
        uint32_t ai = 0;
        uint32_t it = 0;
        bool ok = true;
        for (uint64_t i = 0; i < sched.count && ok; ++i, ++it) {
            uint64_t base;
            int cnt;
            const TcExp* x = tile_at(sched, &one, table, prefix, E, i, base, cnt);
            const int nch = x->nchunks, nkb = x->nkb;
            const int bb = it & 1;
            if (!(ok = wait_bar(&bits_full[bb], (it >> 1) & 1u, sAbort, err, 5, wlim))) break;
            const uint32_t* row = sBits + bb * kTileM * RS + r * RS;
            for (int c = 0; c < nch && ok; ++c)
                for (int kb = 0; kb < nkb; ++kb, ++ai) {
                    const int s = ai % kStagesA;
                    if (!(ok = wait_bar(&a_empty[s], ((ai / kStagesA) & 1u) ^ 1u, sAbort, err, 6, wlim))) break;
                    unsigned char* dst = sA + s * kABytes + (r >> 3) * 1024 + (r & 7) * 128;
                    const uint32_t w2[2] = {row[2 * kb], row[2 * kb + 1]};
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t x = (w2[q >> 2] >> (8 * (q & 3))) & 0xFFu;
                        *reinterpret_cast<uint4*>(dst + ((q ^ (r & 7)) << 4)) = sLut8[x];
                    }
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&a_full[s]);
                }
            __syncwarp();
            if (ok && lane == 0) mbar_arrive(&bits_empty[bb]);
        }
    } else if (warp >= 6 + kExpWarps) {
        // ------------------------------------------------------ generation --
        const int gw = warp - (6 + kExpWarps);
        static_assert(NG * 32 >= kTileM, "exact mode gives every row of a tile its own lane");
        uint32_t it = 0;
        bool ok = true;
        for (uint64_t i = 0; i < sched.count && ok; ++i, ++it) {
            uint64_t base;
            int cnt;
            const TcExp* x = tile_at(sched, &one, table, prefix, E, i, base, cnt);
            const int bb = it & 1;
            if (!(ok = wait_bar(&bits_empty[bb], ((it >> 1) & 1u) ^ 1u, sAbort, err, 7, wlim))) break;
            uint32_t* bits = sBits + bb * kTileM * RS;
            const int kbx = x->kb, nx = x->n, n1x = x->n1, ex = x->exact;
            const uint64_t sx = x->seed, fx = x->first;
            const uint64_t* bx = x->binom;
            if (ex) {
                // exact enumeration: lane j of this warp unranks row gw + NG j on its own
                const int r = gw + NG * lane;
                if (r < kTileM) {
                    uint32_t* row = bits + r * RS;
                    if (r < cnt) lane_exact_row(fx + base + r, nx, n1x, bx, row, 4 * kbx);
                    else for (int q = 0; q < 4 * kbx; ++q) row[q] = 0u;
                }
            } else {
                for (int r = gw; r < kTileM; r += NG) {
                    uint32_t* row = bits + r * RS;
                    if (r < cnt) {
                        if constexpr (MULTI) draw_bits_kb<KB>(kbx, false, sx, fx + base + r, nx, n1x, bx, row, lane);
                        else warp_draw_bits_rk<KB>(one.rk, fx + base + r, nx, n1x, row, lane);
                    } else {
                        for (int q = lane; q < W; q += 32) row[q] = 0u;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bits_full[bb]);
        }
    } else {
        // ------------------------------------------------------- epilogue --
        const int ew = warp;  // 0..3: TMEM lanes 32 ew .. 32 ew + 31
        uint32_t g = 0;
        bool ok = true;
        for (uint64_t i = 0; i < sched.count && ok; ++i) {
            uint64_t base;
            int cnt;
            const TcExp* x = tile_at(sched, &one, table, prefix, E, i, base, cnt);
            const int nch = x->nchunks, dd = x->d;
            float sumsq = 0.f;
            for (int c = 0; c < nch; ++c, ++g) {
                const int buf = g & 1;
                if (!(ok = wait_bar(&acc_full[buf], (g >> 1) & 1u, sAbort, err, 8, wlim))) break;
                tc_fence_after();
                const int rem = dd - c * kChunkN;
                const int N = rem >= kChunkN ? kChunkN : rem;
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * kChunkN);
                for (int c0 = 0; c0 < N; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld32(taddr + (uint32_t)c0, v);
                    tmem_wait_ld();
                    const int lim = N - c0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float x = __uint_as_float(v[j]);
                        if (j < lim) sumsq = fmaf(x, x, sumsq);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
            const int row = 32 * ew + lane;
            const uint64_t off = base + row;
            const float mh = x->c_M * sumsq;
            if (ok && row < cnt) x->Mout[off] = mh;
            // level-0 histogram of the streaming selection (bits [31:20] of M_hat), one atomic
            // per distinct bin of the warp
            unsigned* h0 = x->hist0;
            if (h0 != nullptr) {
                const bool take = ok && row < cnt;
                const unsigned bin = __float_as_uint(mh) >> 20;
                const unsigned mask = __activemask();
                const unsigned peers = __match_any_sync(mask, take ? bin : 0xffffffffu);
                if (take && (__ffs(peers) - 1) == lane) atomicAdd(&h0[bin], (unsigned)__popc(peers));
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

bool make_map(CUtensorMap* m, const __nv_bfloat16* base, int kpad, int d)
{
    return make_map_bf16(m, base, (uint64_t)kpad, (uint64_t)d, (uint32_t)kKBlock, (uint32_t)kChunkN);
}

size_t smem_bytes(int KB, int SB)
{
    const size_t bars = (size_t)(2 * SB + 2 * kStagesA + 9) * 8 + 16;
    return 1024 + (size_t)SB * kBBytes + (size_t)kStagesA * kABytes + 2ull * kTileM * (4 * KB + 1) * 4 + 8 + bars;
}

template <int KB, int SB, int NG>
frr_status launch(frr_ctx* ctx, cudaStream_t stream, int num_sms, const TcExp& one, const TcExp* table,
                  const unsigned long long* prefix, int E, unsigned long long tiles, int* err)
{
    const size_t smem = smem_bytes(KB, SB);
    const unsigned grid = (unsigned)(tiles < (unsigned long long)num_sms ? tiles : (unsigned long long)num_sms);
    if (table == nullptr) {
        FRR_CUDA_TRY(ctx, set_smem_limit(k_balance_tc<KB, SB, NG, false>, (int)smem, ctx->device));
        k_balance_tc<KB, SB, NG, false><<<grid, (6 + kExpWarps + NG) * 32, smem, stream>>>(one, table, prefix, E, tiles, err);
    } else {
        FRR_CUDA_TRY(ctx, set_smem_limit(k_balance_tc<KB, SB, NG, true>, (int)smem, ctx->device));
        k_balance_tc<KB, SB, NG, true><<<grid, (6 + kExpWarps + NG) * 32, smem, stream>>>(one, table, prefix, E, tiles, err);
    }
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

// ---- compiled configurations and their tuning ------------------------------------------
// (KB, SB, NG): Philox blocks per lane of the generating warps, B-operand stages, and
// generating warps per CTA, i.e. how many draws each SM selects concurrently. A CTA has
// 10 + NG warps (at most 32), and the register file gives each thread at most
// 65536 / (32 (10 + NG)) registers, so long draws (large KB) get fewer generating warps.
// Every configuration issues the same MMA sequence for a draw, so all of them produce
// bit-identical M_hat; they differ only in speed, which depends on n (generation cost per
// draw) and d (tensor work per draw).
struct TcCfg {
    int kb, sb, ng;
};
constexpr TcCfg kCfg[] = {
    {1, 4, 10}, {1, 4, 14}, {1, 4, 18}, {1, 4, 22},
    {2, 4, 10}, {2, 4, 14}, {2, 4, 18}, {2, 4, 22},
    {4, 4, 10}, {4, 4, 14}, {4, 4, 18}, {4, 4, 22},
    {8, 4, 8},  {8, 4, 10}, {8, 4, 12},
    {16, 3, 4}, {16, 3, 6},
};
constexpr int kNumCfg = (int)(sizeof(kCfg) / sizeof(kCfg[0]));

using LaunchFn = frr_status (*)(frr_ctx*, cudaStream_t, int, const TcExp&, const TcExp*, const unsigned long long*, int,
                                unsigned long long, int*);

template <size_t... I>
constexpr std::array<LaunchFn, sizeof...(I)> launch_table(std::index_sequence<I...>)
{
    return {{&launch<kCfg[I].kb, kCfg[I].sb, kCfg[I].ng>...}};
}
constexpr std::array<LaunchFn, kNumCfg> kLaunch = launch_table(std::make_index_sequence<kNumCfg>{});

// built-in choice per KB (measured on B300 with d up to 1000), used until a shape class is tuned
int default_cfg(int kb)
{
    switch (kb) {
        case 1: return 3;
        case 2: return 7;
        case 4: return 11;
        case 8: return 13;
        case 16: return 16;
        default: return -1;
    }
}

std::mutex g_tune_mu;
std::map<std::array<int, 4>, int> g_tuned;  // (device, KB, covariate chunks, batched) -> configuration

int chosen_cfg(int device, int kb, int nch, bool multi)
{
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        const auto it = g_tuned.find({device, kb, nch, multi ? 1 : 0});
        if (it != g_tuned.end()) return it->second;
    }
    return default_cfg(kb);
}

void remember_cfg(int device, int kb, int nch, bool multi, int cfg)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[{device, kb, nch, multi ? 1 : 0}] = cfg;
}

bool tuned_already(int device, int kb, int nch, bool multi)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return g_tuned.count({device, kb, nch, multi ? 1 : 0}) != 0;
}

frr_status launch_cfg(int cfg, frr_ctx* ctx, cudaStream_t stream, int num_sms, const TcExp& one, const TcExp* table,
                      const unsigned long long* prefix, int E, unsigned long long tiles, int* err)
{
    if (cfg < 0 || cfg >= kNumCfg) return FRR_E_UNSUPPORTED;
    return kLaunch[(size_t)cfg](ctx, stream, num_sms, one, table, prefix, E, tiles, err);
}

// Times configuration `cfg` (one warm-up launch, then the fastest of `reps`); run(cfg)
// enqueues one launch on `stream`.
template <typename Run>
frr_status time_cfg(frr_ctx* ctx, cudaStream_t stream, int cfg, int reps, Run&& run, float* ms_out)
{
    cudaEvent_t e0, e1;
    FRR_CUDA_TRY(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        FRR_CUDA_TRY(ctx, cudaGetLastError());
    }
    frr_status s = run(cfg);
    float best = INFINITY;
    for (int r = 0; r < reps && s == FRR_OK; ++r) {
        cudaEventRecord(e0, stream);
        s = run(cfg);
        cudaEventRecord(e1, stream);
        if (s == FRR_OK && cudaEventSynchronize(e1) != cudaSuccess) s = FRR_E_CUDA;
        float ms = 0.f;
        if (s == FRR_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == FRR_E_CUDA) {
        cudaGetLastError();
        ctx->failed = true;
    }
    *ms_out = best;
    return s;
}

}  // namespace

// Fills the experiment descriptor of a prepared context for draws [first, first + B).
frr_status tc_describe(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout, TcExp* x)
{
    if (!ctx->maps_ready) {
        if (!make_map(&ctx->map_hi, ctx->Zhi, ctx->kpad, (int)ctx->d) ||
            !make_map(&ctx->map_lo, ctx->Zlo, ctx->kpad, (int)ctx->d))
            return FRR_E_CUDA;
        ctx->maps_ready = true;
    }
    x->map_hi = ctx->map_hi;
    x->map_lo = ctx->map_lo;
    x->binom = ctx->binom;
    x->Mout = Mout;
    x->seed = seed;
    philox_round_keys(seed, x->rk);
    x->first = first;
    x->B = B;
    x->c_M = (float)ctx->c_M;
    x->n = (int)ctx->n;
    x->n1 = (int)ctx->n1;
    x->d = (int)ctx->d;
    x->kb = ctx->kb;
    x->nkb = ctx->kused / kKBlock;
    x->nchunks = ceil_div(ctx->d, kChunkN);
    x->exact = exact ? 1 : 0;
    x->skip_tma = 0;
    x->wait_cycles = 0;
    x->hist0 = nullptr;
    return FRR_OK;
}

frr_status balance_tc_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout,
                             unsigned* hist0)
{
    if (B == 0) return FRR_OK;
    TcExp one;
    FRR_TRY(tc_describe(ctx, seed, exact, first, B, Mout, &one));
    one.hist0 = hist0;
    const unsigned long long tiles = (B + kTileM - 1) / kTileM;
    const int cfg = chosen_cfg(ctx->device, ctx->kb, one.nchunks, false);
    return launch_cfg(cfg, ctx, ctx->stream, ctx->num_sms, one, nullptr, nullptr, 1, tiles, ctx->dev_counters + 12);
}

// One persistent launch over E experiments: `table` (device, E entries) describes them,
// `prefix` (device, E + 1 entries) holds the first global tile of each. kbmax bounds their
// Philox blocks per lane and nchmax their covariate chunks; the launch goes to `stream`.
// Errors from bounded waits go to *err (device).
frr_status balance_tc_batch_launch(frr_ctx* owner, cudaStream_t stream, const TcExp* table,
                                   const unsigned long long* prefix, int E, unsigned long long tiles, int kbmax,
                                   int nchmax, int* err)
{
    if (tiles == 0) return FRR_OK;
    TcExp unused{};
    const int cfg = chosen_cfg(owner->device, kbmax, nchmax, true);
    return launch_cfg(cfg, owner, stream, owner->num_sms, unused, table, prefix, E, tiles, err);
}

// Times every configuration for kbmax on a (probe) batch described like the launch above
// and makes the fastest the choice for batches of this shape class.
frr_status balance_tc_batch_tune(frr_ctx* owner, cudaStream_t stream, const TcExp* table,
                                 const unsigned long long* prefix, int E, unsigned long long tiles, int kbmax,
                                 int nchmax, int* err)
{
    if (tiles == 0) return FRR_OK;
    // a class is timed once per process (frr_autotune re-times a context's class on request)
    if (tuned_already(owner->device, kbmax, nchmax, true)) return FRR_OK;
    TcExp unused{};
    int best = -1;
    float best_ms = INFINITY;
    for (int c = 0; c < kNumCfg; ++c) {
        if (kCfg[c].kb != kbmax) continue;
        float ms = INFINITY;
        FRR_TRY(time_cfg(owner, stream, c, 2,
                         [&](int cfg) {
                             return launch_cfg(cfg, owner, stream, owner->num_sms, unused, table, prefix, E, tiles,
                                               err);
                         },
                         &ms));
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    if (best < 0) return FRR_E_UNSUPPORTED;
    remember_cfg(owner->device, kbmax, nchmax, true, best);
    return FRR_OK;
}

}  // namespace frr

using namespace frr;

extern "C" frr_status frr_autotune(frr_ctx* ctx, uint64_t B_probe, frr_tune_result* out)
{
    if (!ctx || !out || B_probe > (1ull << 24)) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (ctx->opts.precision != FRR_SPLIT_BF16) return FRR_E_UNSUPPORTED;
    if (B_probe == 0) B_probe = 8ull * kTileM * (uint64_t)ctx->num_sms;
    std::memset(out, 0, sizeof(*out));
    const size_t bytes = (size_t)B_probe * sizeof(float);
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->Mhat), &ctx->Mhat_bytes, 2 * bytes));
    float* ref = ctx->Mhat;
    float* cmp = ctx->Mhat + B_probe;
    TcExp one;
    constexpr uint64_t kProbeSeed = 0x7E57C0DEull;
    FRR_TRY(tc_describe(ctx, kProbeSeed, false, 0, B_probe, ref, &one));
    const unsigned long long tiles = (B_probe + kTileM - 1) / kTileM;
    std::vector<float> h_ref(B_probe), h_cmp(B_probe);
    out->kb = ctx->kb;
    out->chunks = one.nchunks;
    int best = -1, best_i = -1;
    float best_ms = INFINITY;
    for (int c = 0; c < kNumCfg; ++c) {
        if (kCfg[c].kb != ctx->kb || out->candidates >= FRR_TUNE_MAX) continue;
        const int i = out->candidates++;
        one.Mout = (i == 0) ? ref : cmp;
        float ms = INFINITY;
        FRR_TRY(time_cfg(ctx, ctx->stream, c, 3,
                         [&](int cfg) {
                             return launch_cfg(cfg, ctx, ctx->stream, ctx->num_sms, one, nullptr, nullptr, 1, tiles,
                                               ctx->dev_counters + 12);
                         },
                         &ms));
        FRR_TRY(take_device_error(ctx));
        // every configuration must reproduce the first one's M_hat bit for bit
        FRR_TRY(copy_out(ctx, i == 0 ? h_ref.data() : h_cmp.data(), one.Mout, bytes));
        if (i > 0 && std::memcmp(h_ref.data(), h_cmp.data(), bytes) != 0) return FRR_E_MISMATCH;
        out->ng[i] = kCfg[c].ng;
        out->sb[i] = kCfg[c].sb;
        out->ms[i] = ms;
        if (ms < best_ms) { best_ms = ms; best = c; best_i = i; }
    }
    if (best < 0) return FRR_E_UNSUPPORTED;
    out->chosen = best_i;
    remember_cfg(ctx->device, ctx->kb, one.nchunks, false, best);
    return FRR_OK;
}

extern "C" frr_status frr_test_wait_expiry(frr_ctx* ctx, uint64_t wait_cycles)
{
    if (!ctx) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (ctx->opts.precision != FRR_SPLIT_BF16) return FRR_E_UNSUPPORTED;
    if (wait_cycles < 10000) wait_cycles = 10000;
    if (wait_cycles > kWaitCycles) wait_cycles = kWaitCycles;
    // one tile of 128 draws per SM; the covariate tiles never arrive, so the first MMA wait
    // expires, the CTA raises its abort flag and every other role returns through its own
    // bounded wait; TMEM is released at the kernel's end as on every exit
    const uint64_t B = (uint64_t)kTileM * (uint64_t)ctx->num_sms;
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->Mhat), &ctx->Mhat_bytes, (size_t)B * sizeof(float)));
    TcExp one;
    FRR_TRY(tc_describe(ctx, 1, false, 0, B, ctx->Mhat, &one));
    one.skip_tma = 1;
    one.wait_cycles = wait_cycles;
    const int cfg = chosen_cfg(ctx->device, ctx->kb, one.nchunks, false);
    FRR_TRY(launch_cfg(cfg, ctx, ctx->stream, ctx->num_sms, one, nullptr, nullptr, 1, (B + kTileM - 1) / kTileM,
                       ctx->dev_counters + 12));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return take_device_error(ctx);
}
