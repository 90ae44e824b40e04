// frr_distance.cu -- pairwise Euclidean distances on the tensor cores (Sec. 4,
// fast_distance): D_ij = ||x_i - y_j|| = sqrt(||x_i||^2 + ||y_j||^2 - 2 x_i . y_j).
//
// The cross term is a dense contraction over d, so it runs as one tcgen05 GEMM. FP32
// inputs are split into BF16 parts h = bf16(v), l = bf16(v - h) and the three products
// that carry the precision are folded into a single K dimension of 3 dp (dp = d rounded
// up to 64):
//   A row i = [x_h | x_h | x_l],   B row j = [y_h | y_l | y_h],   A_i . B_j = x.y - x_l y_l - e,
// with |x - x_h - x_l| <= 2^-18 |x| per element. Squared norms come from the FP32 values
// (a compensated sum, about as accurate as twice the FP32 precision). The epilogue reads the accumulator from TMEM, adds the norms, clamps
// at 0, takes the square root (unless the squared distance was asked for) and stages
// 32 x 32 blocks in shared memory for TMA stores (direct stores when the output rows are
// not 16-byte aligned).
//
// k_distance_tc: one persistent CTA per SM over 128 x 256 output tiles (grouped by
// bands of tile rows so that the B rows stay in L2). Warp roles:
//   warps 0-7  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one output row per
//              thread) and the column half w / 4 of the 256 columns;
//   warp 8     TMA producer: A (128 x 64) and B (256 x 64) K blocks, 128-byte swizzle,
//              into a 4-stage ring;
//   warp 9     TMEM allocator (512 columns: two 256-column accumulators) and MMA issuer.
// Every mbarrier wait is bounded; on expiry the CTA records an error word, drains its
// own TMA copies, frees TMEM and returns.
#include "frr_internal.cuh"

#include <cuda.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "frr_tc_ptx.cuh"

namespace frr {
using namespace tc;
namespace {

constexpr int kDM = 128;                       // rows of X per tile (TMEM lanes)
constexpr int kDN = 256;                       // rows of Y per tile (accumulator columns)
constexpr int kDK = 64;                        // K elements per stage (128 bytes of BF16)
constexpr int kDStages = 4;
constexpr int kDABytes = kDM * kDK * 2;        // 16 KiB
constexpr int kDBBytes = kDN * kDK * 2;        // 32 KiB
constexpr int kDStageBytes = kDABytes + kDBBytes;
constexpr int kDEpiWarps = 8;
constexpr int kDThreads = (kDEpiWarps + 2) * 32;
constexpr int kDGroup = 32;                    // tile rows per band of the tile order (4096 rows of X)
constexpr int kDOutBytes = 32 * 32 * 4;        // per epilogue warp: 32 rows x 32 columns staged for a TMA store
constexpr size_t kDSmem = 1024 + (size_t)kDStages * kDStageBytes + (size_t)kDEpiWarps * kDOutBytes + 256;

// Error-free transformations (Knuth's TwoSum; the FMA product error), used for the
// squared norms in the manner of Ogita, Rump and Oishi's Dot2 (SIAM J. Sci. Comput. 26,
// 2005): the sum of squares is carried as an unevaluated pair (s, c), about as accurate as
// a sum in twice the FP32 precision, and rounded once at the end.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Split rows into the K-major BF16 operands (rows x 3 dp) and the squared norms, one warp
// per row: rows [0, n) of X into A with layout [h | h | l], rows [0, m) of Y into B with
// layout [h | l | h]; lane l handles elements 4l + 128 i (four per 16-byte load when the
// rows are 16-byte aligned). The same launch zeroes the column norms' padding [m, mpad)
// and the error word, so a call needs no memsets.
// BF16 parts h = bf16(x), l = bf16(x - h) of four values, packed as two 8-byte words
__device__ __forceinline__ void split4(const float (&x)[4], uint2& hw, uint2& lw)
{
    __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h[q] = __float2bfloat16_rn(x[q]);
        l[q] = __float2bfloat16_rn(x[q] - __bfloat162float(h[q]));
    }
    memcpy(&hw, h, 8);
    memcpy(&lw, l, 8);
}

__global__ void __launch_bounds__(256) k_dist_prep(const float* __restrict__ X, int64_t n, const float* __restrict__ Y,
                                                   int64_t m, int64_t mpad, int d, int dp, int vec,
                                                   __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B,
                                                   float* __restrict__ nx, float* __restrict__ ny, int* __restrict__ err)
{
    const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
    if (w >= n + m) {
        // the padding of the column norms, one entry per thread of the trailing blocks
        const int64_t pidx = m + (w - n - m) * 32 + lane;
        if (pidx < mpad) ny[pidx] = 0.0f;
        return;
    }
    const bool side_b = w >= n;
    const int64_t r = side_b ? w - n : w;
    const float* v = (side_b ? Y : X) + r * (int64_t)d;
    __nv_bfloat16* o = (side_b ? B : A) + r * (int64_t)(3 * dp);
    float s = 0.f, c = 0.f;
    for (int k = 4 * lane; k < dp; k += 128) {
        float x[4];
        if (vec && k + 4 <= d) {
            const float4 t = *reinterpret_cast<const float4*>(v + k);
            x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = k + q < d ? v[k + q] : 0.0f;
        }
        // [h | h | l] for X, [h | l | h] for Y
        uint2 hw, lw;
        split4(x, hw, lw);
        *reinterpret_cast<uint2*>(o + k) = hw;
        *reinterpret_cast<uint2*>(o + dp + k) = side_b ? lw : hw;
        *reinterpret_cast<uint2*>(o + 2 * dp + k) = side_b ? hw : lw;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float p = x[q] * x[q];
            const float pe = fmaf(x[q], x[q], -p);
            float t, e;
            two_sum(s, p, t, e);
            s = t;
            c += e + pe;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, off);
        const float co = __shfl_xor_sync(0xffffffffu, c, off);
        float t, q;
        two_sum(s, so, t, q);
        s = t;
        c += co + q;
    }
    if (lane == 0) (side_b ? ny : nx)[r] = s + c;
}

__device__ __forceinline__ void dist_tile_of(uint64_t t, int ntn, int ntm, int& tm, int& tn)
{
    // bands of kDGroup tile rows; inside a band, tile rows vary fastest
    const uint64_t per_band = (uint64_t)kDGroup * ntn;
    const int band = (int)(t / per_band);
    const int first = band * kDGroup;
    const int rows = (ntm - first) < kDGroup ? (ntm - first) : kDGroup;
    const uint64_t in = t - (uint64_t)band * per_band;
    tm = first + (int)(in % rows);
    tn = (int)(in / rows);
}

__global__ void __launch_bounds__(kDThreads, 1)
k_distance_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              const __grid_constant__ CUtensorMap mapD, const float* __restrict__ nx, const float* __restrict__ ny,
              int n, int m, int nkb, int squared, int tma_out, int vec4, float* __restrict__ D, int* err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* sOut = reinterpret_cast<float*>(smem + kDStages * kDStageBytes);   // kDEpiWarps x 32 x 32, 128B-swizzled
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kDStages * kDStageBytes + kDEpiWarps * kDOutBytes);
    uint64_t* full = bar;
    uint64_t* empty = full + kDStages;
    uint64_t* acc_full = empty + kDStages;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* mma_done = acc_empty + 2;
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntm = (n + kDM - 1) / kDM, ntn = (m + kDN - 1) / kDN;
    const uint64_t tiles = (uint64_t)ntm * ntn;

    if (tid == 0) {
        for (int s = 0; s < kDStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) { mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], kDEpiWarps); }
        mbar_init(mma_done, 1);
        *sAbort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kDEpiWarps + 1) {
        tmem_alloc(sTmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *sTmem;

    if (warp == kDEpiWarps) {
        // ------------------------------------------------------------ TMA --
        if (lane == 0) {
            uint32_t i = 0;
            bool ok = true;
            for (uint64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int tm, tn;
                dist_tile_of(t, ntn, ntm, tm, tn);
                for (int kb = 0; kb < nkb; ++kb, ++i) {
                    const int s = i % kDStages;
                    if (!(ok = wait_bar(&empty[s], ((i / kDStages) & 1u) ^ 1u, sAbort, err, 11))) break;
                    unsigned char* st = smem + s * kDStageBytes;
                    mbar_arrive_expect_tx(&full[s], kDStageBytes);
                    tma_load_2d(st, &mapA, &full[s], kb * kDK, tm * kDM);
                    tma_load_2d(st + kDABytes, &mapB, &full[s], kb * kDK, tn * kDN);
                }
            }
            if (!ok) {
                const uint32_t from = i > (uint32_t)kDStages ? i - kDStages : 0u;
                for (uint32_t j = from; j < i; ++j) {
                    const unsigned long long t0 = clock64();
                    while (!mbar_try_wait(&full[j % kDStages], (j / kDStages) & 1u) && clock64() - t0 < kWaitCycles) {}
                }
            }
        }
    } else if (warp == kDEpiWarps + 1) {
        // ------------------------------------------------------------ MMA --
        if (lane == 0) {
            uint32_t i = 0, g = 0;
            bool ok = true;
            const uint32_t idesc = idesc_bf16(kDM, kDN);
            for (uint64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++g) {
                const int buf = g & 1;
                if (!(ok = wait_bar(&acc_empty[buf], ((g >> 1) & 1u) ^ 1u, sAbort, err, 12))) break;
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(buf * kDN);
                for (int kb = 0; kb < nkb; ++kb, ++i) {
                    const int s = i % kDStages;
                    if (!(ok = wait_bar(&full[s], (i / kDStages) & 1u, sAbort, err, 13))) break;
                    tc_fence_after();
                    const uint64_t adesc = sdesc_sw128(smem_u32(smem + s * kDStageBytes));
                    const uint64_t bdesc = sdesc_sw128(smem_u32(smem + s * kDStageBytes + kDABytes));
#pragma unroll
                    for (int k = 0; k < kDK / 16; ++k)
                        umma_bf16(dt, adesc + 2u * k, bdesc + 2u * k, idesc, (kb | k) != 0 ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&acc_full[buf]);
            }
            umma_commit(mma_done);
            const unsigned long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {}
        }
    } else {
        // ------------------------------------------------------- epilogue --
        const int quarter = warp & 3, half = warp >> 2;
        uint32_t g = 0;
        bool ok = true;
        for (uint64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++g) {
            int tm, tn;
            dist_tile_of(t, ntn, ntm, tm, tn);
            const int buf = g & 1;
            if (!(ok = wait_bar(&acc_full[buf], (g >> 1) & 1u, sAbort, err, 14))) break;
            tc_fence_after();
            const int row0 = tm * kDM + 32 * quarter;
            const int row = row0 + lane;
            const float nrow = row < n ? nx[row] : 0.0f;
            float* drow = D + (size_t)(row < n ? row : 0) * (size_t)m;
            float* sbuf = sOut + warp * (kDOutBytes / 4);
            for (int c0 = half * (kDN / 2); c0 < (half + 1) * (kDN / 2); c0 += 32) {
                const int col0 = tn * kDN + c0;
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(tmem_base + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * kDN + c0), v);
                tmem_wait_ld();
                if (row0 >= n || col0 >= m) continue;   // warp-uniform: nothing of this chunk is stored
                // the norms of the 32 columns (padded with zeros past m), as 8 broadcast loads
                float ncol[32];
                const float4* ny4 = reinterpret_cast<const float4*>(ny + col0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 t4 = __ldg(ny4 + q);
                    ncol[4 * q] = t4.x; ncol[4 * q + 1] = t4.y; ncol[4 * q + 2] = t4.z; ncol[4 * q + 3] = t4.w;
                }
                float out[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float d2 = fmaf(-2.0f, __uint_as_float(v[j]), nrow + ncol[j]);
                    d2 = fmaxf(d2, 0.0f);
                    out[j] = squared ? d2 : sqrtf(d2);
                }
                if (tma_out) {
                    // stage row `lane` (16-byte chunk q at q ^ (lane % 8), the 128-byte swizzle)
                    // and let one TMA store write the 32 x 32 block, clipped to n x m
                    if (lane == 0) bulk_wait_read();
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(sbuf + lane * 32 + 4 * (q ^ (lane & 7))) =
                            make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&mapD, sbuf, col0, row0);
                        bulk_commit();
                    }
                } else if (row < n) {
                    if (vec4 && col0 + 32 <= m) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4*>(drow + col0 + j) =
                                make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < m) drow[col0 + j] = out[j];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    }

    if (warp < kDEpiWarps && lane == 0) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == kDEpiWarps + 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

}  // namespace
}  // namespace frr

using namespace frr;

namespace {

struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

// The operand temporaries come from a pool per device that keeps its memory after the
// call (release threshold: never), so repeated calls do not map and unmap it again.
cudaMemPool_t dist_pool(int dev)
{
    static std::mutex mu;
    static std::unordered_map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
    return pool;
}

frr_status dist_alloc(DevBuf& b, size_t bytes, cudaStream_t s, cudaMemPool_t pool = nullptr)
{
    b.s = s;
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&b.p, bytes ? bytes : 16, pool, s)
                               : cudaMallocAsync(&b.p, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e == cudaErrorMemoryAllocation ? FRR_E_NOMEM : FRR_E_CUDA;
    }
    return FRR_OK;
}

#define DIST_CUDA(expr)                                                                 \
    do {                                                                                \
        const cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return _e == cudaErrorMemoryAllocation ? FRR_E_NOMEM : FRR_E_CUDA;          \
        }                                                                               \
    } while (0)

}  // namespace

extern "C" frr_status frr_fast_distance(const float* X, int64_t n, const float* Y, int64_t m, int64_t d, int squared,
                                        float* D_out, void* cuda_stream)
{
    if (X == nullptr || D_out == nullptr || n < 1 || d < 1) return FRR_E_ARG;
    if (Y == nullptr) m = n;
    if (m < 1) return FRR_E_ARG;
    if (n > (1ll << 30) || m > (1ll << 30) || d > (1ll << 20)) return FRR_E_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    DIST_CUDA(cudaGetDevice(&dev));
    DIST_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    const int dp = (int)((d + kDK - 1) / kDK) * kDK;
    const int64_t kp = 3ll * dp;
    // every temporary comes from the library's per-device pool, which keeps its memory
    // mapped between calls (a pool that returns it at each synchronisation maps it again on
    // the next call)
    cudaMemPool_t pool = dist_pool(dev);
    if (pool == nullptr) return FRR_E_CUDA;
    DevBuf xin, yin, A, B, nX, nY, Dd, errb;
    const float* Xd = X;
    const float* Yd = Y;
    if (!is_device_ptr(X)) {
        FRR_TRY(dist_alloc(xin, (size_t)n * d * sizeof(float), s, pool));
        DIST_CUDA(cudaMemcpyAsync(xin.p, X, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, s));
        Xd = static_cast<const float*>(xin.p);
    }
    if (Y == nullptr) {
        Yd = Xd;
    } else if (!is_device_ptr(Y)) {
        FRR_TRY(dist_alloc(yin, (size_t)m * d * sizeof(float), s, pool));
        DIST_CUDA(cudaMemcpyAsync(yin.p, Y, (size_t)m * d * sizeof(float), cudaMemcpyHostToDevice, s));
        Yd = static_cast<const float*>(yin.p);
    }
    FRR_TRY(dist_alloc(A, (size_t)n * kp * 2, s, pool));
    FRR_TRY(dist_alloc(B, (size_t)m * kp * 2, s, pool));
    FRR_TRY(dist_alloc(nX, (size_t)n * sizeof(float), s, pool));
    const int64_t mpad = (m + kDN - 1) / kDN * kDN;   // column norms padded with zeros to whole tiles
    FRR_TRY(dist_alloc(nY, (size_t)mpad * sizeof(float), s, pool));
    FRR_TRY(dist_alloc(errb, sizeof(int), s, pool));
    float* Dw = D_out;
    const bool dev_out = is_device_ptr(D_out);
    if (!dev_out) {
        FRR_TRY(dist_alloc(Dd, (size_t)n * m * sizeof(float), s, pool));
        Dw = static_cast<float*>(Dd.p);
    }
    // one launch splits both operands, zeroes the norm padding and the error word
    const int vec = ((d & 3) == 0 && (reinterpret_cast<uintptr_t>(Xd) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(Yd) & 15u) == 0) ? 1 : 0;
    const int64_t prep_warps = n + m + (mpad - m + 31) / 32;
    k_dist_prep<<<(unsigned)((prep_warps + 7) / 8), 256, 0, s>>>(Xd, n, Yd, m, mpad, (int)d, dp, vec,
                                                                static_cast<__nv_bfloat16*>(A.p),
                                                                static_cast<__nv_bfloat16*>(B.p),
                                                                static_cast<float*>(nX.p), static_cast<float*>(nY.p),
                                                                static_cast<int*>(errb.p));
    DIST_CUDA(cudaGetLastError());

    CUtensorMap mapA, mapB, mapD;
    if (!make_map_bf16(&mapA, A.p, (uint64_t)kp, (uint64_t)n, kDK, kDM)) return FRR_E_CUDA;
    if (!make_map_bf16(&mapB, B.p, (uint64_t)kp, (uint64_t)m, kDK, kDN)) return FRR_E_CUDA;
    DIST_CUDA(set_smem_limit(k_distance_tc, (int)kDSmem, dev));
    const uint64_t tiles = (uint64_t)((n + kDM - 1) / kDM) * (uint64_t)((m + kDN - 1) / kDN);
    const unsigned grid = (unsigned)(tiles < (uint64_t)sms ? tiles : (uint64_t)sms);
    // 16-byte row stores, and TMA stores, need m % 4 == 0 and a 16-byte aligned output
    const int vec4 = ((m & 3) == 0 && (reinterpret_cast<uintptr_t>(Dw) & 15u) == 0) ? 1 : 0;
    const int tma_out = vec4 && make_map_f32(&mapD, Dw, (uint64_t)m, (uint64_t)n, 32, 32) ? 1 : 0;
    if (!tma_out) memset(&mapD, 0, sizeof(mapD));
    k_distance_tc<<<grid, kDThreads, kDSmem, s>>>(mapA, mapB, mapD, static_cast<const float*>(nX.p),
                                                  static_cast<const float*>(nY.p), (int)n, (int)m, (int)(kp / kDK),
                                                  squared ? 1 : 0, tma_out, vec4, Dw, static_cast<int*>(errb.p));
    DIST_CUDA(cudaGetLastError());
    if (!dev_out)
        DIST_CUDA(cudaMemcpyAsync(D_out, Dw, (size_t)n * m * sizeof(float), cudaMemcpyDeviceToHost, s));
    int herr = 0;
    DIST_CUDA(cudaMemcpyAsync(&herr, errb.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DIST_CUDA(cudaStreamSynchronize(s));
    return herr != 0 ? FRR_E_TIMEOUT : FRR_OK;
}
