// frr_balance_f32.cu -- plain FP32 SIMT balance check (the CUDA-core path).
//
// Hotelling T^2 of each draw b with whitened covariates (Sec. 2.2, 2.3):
//   s_b = w_b^T Zc (1 x d),  M_b = n / (n1 n0) * ||s_b||^2.
// A CTA takes 128 consecutive draws: its 8 warps regenerate their bit rows
// into shared memory (frr_gen.cuh), then the CTA sweeps the FP32 covariates
// (K-order rows, 32 rows x 128 columns per shared-memory stage) and each
// thread accumulates an 8-draw x 8-column register tile with predicated adds
// (w is 0/1). Squares are summed per thread across column tiles and reduced
// over the 16 threads sharing the draws. The assignment matrix never leaves
// shared memory.
#include "frr_internal.cuh"
#include "frr_gen.cuh"

namespace frr {
namespace {

constexpr int TD = 128;     // draws per CTA
constexpr int NT = 256;     // threads per CTA

template <int KB>
__global__ void __launch_bounds__(NT, 2)
k_balance_f32(const float* __restrict__ Z32, int dpad32, int kused, int n, int n1, float c_M, uint64_t seed,
              int exact, const uint64_t* __restrict__ binom, uint64_t first, uint64_t B, float* __restrict__ Mout)
{
    constexpr int W = 4 * KB;
    constexpr int RS = W + 1;  // odd row stride: the two draw rows a warp reads sit in different banks
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* zs = reinterpret_cast<float4*>(smem_raw);                         // 32 rows x 32 float4
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw + 32 * 32 * sizeof(float4));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t tile_off = (uint64_t)blockIdx.x * TD;
    if (exact) {
        // exact enumeration: one colex rank per thread
        static_assert(NT >= TD, "one thread per draw");
        if (threadIdx.x < TD) {
            uint32_t* row = bits + threadIdx.x * RS;
            if (tile_off + threadIdx.x < B) lane_exact_row(first + tile_off + threadIdx.x, n, n1, binom, row, W);
            else for (int q = 0; q < W; ++q) row[q] = 0u;
        }
    } else {
        for (int t = warp; t < TD; t += NT / 32) {
            uint32_t* row = bits + t * RS;
            if (tile_off + t < B) {
                warp_draw_bits<KB>(false, seed, first + tile_off + t, n, n1, binom, row, lane);
            } else {
                for (int q = lane; q < W; q += 32) row[q] = 0u;
            }
        }
    }
    __syncthreads();

    // thread (ty, tx): draws ty + 16 i (i < 8), columns 4tx..4tx+3 and 64+4tx..64+4tx+3 of the tile
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float sumsq[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) sumsq[i] = 0.f;

    for (int c0 = 0; c0 < dpad32; c0 += 128) {
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[i][c] = 0.f;

        for (int m = 0; m < kused / 32; ++m) {
            __syncthreads();
#pragma unroll
            for (int e = threadIdx.x; e < 32 * 32; e += NT) {
                const int r = e >> 5, c4 = e & 31;
                zs[e] = reinterpret_cast<const float4*>(Z32 + (size_t)(32 * m + r) * dpad32 + c0)[c4];
            }
            __syncthreads();
            uint32_t bw[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) bw[i] = bits[(ty + 16 * i) * RS + m];
#pragma unroll 4
            for (int u = 0; u < 32; ++u) {
                const float4 za = zs[u * 32 + tx];
                const float4 zb = zs[u * 32 + 16 + tx];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if ((bw[i] >> u) & 1u) {
                        acc[i][0] += za.x; acc[i][1] += za.y; acc[i][2] += za.z; acc[i][3] += za.w;
                        acc[i][4] += zb.x; acc[i][5] += zb.y; acc[i][6] += zb.z; acc[i][7] += zb.w;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int c = 0; c < 8; ++c) sumsq[i] += acc[i][c] * acc[i][c];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) sumsq[i] += __shfl_xor_sync(kFull, sumsq[i], off);
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int t = ty + 16 * i;
            if (tile_off + t < B) Mout[tile_off + t] = c_M * sumsq[i];
        }
    }
}

template <int KB>
frr_status launch_kb(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout)
{
    const size_t smem = 32 * 32 * sizeof(float4) + (size_t)TD * (4 * KB + 1) * sizeof(uint32_t);
    FRR_CUDA_TRY(ctx, set_smem_limit(k_balance_f32<KB>, (int)smem, ctx->device));
    const uint64_t tiles = (B + TD - 1) / TD;
    k_balance_f32<KB><<<(unsigned)tiles, NT, smem, ctx->stream>>>(ctx->Z32, ctx->dpad32, ctx->kused, (int)ctx->n,
                                                                  (int)ctx->n1, (float)ctx->c_M, seed, exact ? 1 : 0,
                                                                  ctx->binom, first, B, Mout);
    FRR_CUDA_TRY(ctx, cudaGetLastError());
    return FRR_OK;
}

}  // namespace

frr_status balance_f32_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout)
{
    if (B == 0) return FRR_OK;
    switch (ctx->kb) {
        case 1: return launch_kb<1>(ctx, seed, exact, first, B, Mout);
        case 2: return launch_kb<2>(ctx, seed, exact, first, B, Mout);
        case 4: return launch_kb<4>(ctx, seed, exact, first, B, Mout);
        case 8: return launch_kb<8>(ctx, seed, exact, first, B, Mout);
        case 16: return launch_kb<16>(ctx, seed, exact, first, B, Mout);
        default: return FRR_E_UNSUPPORTED;
    }
}

}  // namespace frr
