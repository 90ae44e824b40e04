// frr_prep_tc.cu -- the parts of the preparation (Sec. 2.2) that run as exact integer sums
// on the tensor cores when frr_opts.prep = FRR_PREP_TENSOR: the covariance S = Xc^T Xc /
// (n - 1), and the updates of the forward substitution Zc = Xc L^{-T} across blocks of 256
// columns.
//
// Digit products. Each operand vector (a centred column of Xc for the covariance; a row of
// the working Zc or of L over a kFwdBlock-column block for the forward substitution) is scaled by
// a power of two, 2^(55 - e) with every entry below 2^e in magnitude, and rounded to
// integers v (|v| <= 2^55), which are cut into eight balanced base-128 digits, v = sum_{s<8}
// g_s 128^(7-s), g_1..g_7 in [-64, 63] and |g_0| <= 65; every digit is exact in BF16. For
// two vectors a, b
//   sum_i v_a,i v_b,i = sum_{s,t} P_st 2^(7(14-s-t)),   P_st = sum_i g_s(a, i) g_t(b, i),
// and the pairs with s + t <= 7 carry it to 2^-56 of its largest possible value. Over a
// block of 512 terms every P_st is an integer below 2^22 in magnitude (512 * 65^2), so the
// tensor cores' FP32 accumulation of the digit products is exact. P_st 2^(7(14-s-t) - 59)
// is added into one int64 per element (exactly for s + t <= 5, rounded to nearest for the
// last two levels, an error of at most one unit of 2^59 per term); the sum is at most
// 2048 2^110 / 2^59 < 2^63 in magnitude. The element is that sum times 2^(59 + e_a + e_b -
// 110), converted to FP64 once.
//
// Work units of (128 x 128 tile of the output, a quarter of the 36 digit pairs) are taken
// by persistent CTAs; each unit adds its partial sums into the job's int64 sums with atomics
// (integer addition: the order does not matter), and a last kernel converts the sums.
// Warps 0-15 epilogue (warp w: TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..), warp 16
// TMA (per K block of 64 terms: the two 128-row digit tiles), warp 17 MMA (M = 128, N = 128,
// K = 16), four 128-column accumulators in TMEM so that the epilogue of one pair overlaps
// the MMAs of the next.
#include "frr_internal.cuh"

#include <algorithm>
#include "frr_exact.cuh"
#include "frr_tc_ptx.cuh"

namespace frr {
using namespace tc;
using namespace exact;
namespace {

constexpr int kDig = 8;            // digits per covariate
constexpr int kDigBits = 7;
constexpr int kPairs = 36;         // s + t <= 7
constexpr int kGroups = 4;         // pair quarters (work units per tile)
constexpr int kPairsPerGroup = kPairs / kGroups;
constexpr int kShift = 59;         // the int64 sums hold sum_i v_ij v_ik / 2^59
constexpr int kT = 128;            // tile edge (rows j = MMA M, columns k = MMA N)
constexpr int kKB = 64;            // rows i per K block (one 128-byte swizzled row per tile row)
constexpr int kChunkKB = 8;        // K blocks per exact accumulation (512 rows)
constexpr int kStages = 5;
constexpr int kTileBytes = kT * kKB * 2;   // 16 KiB per operand tile
constexpr int kStageBytes = 2 * kTileBytes;
constexpr int kAccBufs = 4;
constexpr int kEpiWarps = 16;
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr int kStatusTimeout = 2;  // the preparation's status bit of an expired bounded wait
static_assert(kPairs % kGroups == 0, "equal pair groups");
static_assert(kFwdBlock % 64 == 0 && kFwdBlock <= kChunkKB * 64, "forward blocks of whole K blocks, one exact chunk");
static_assert(kChunkKB * kKB * 65 * 65 < (1 << 22), "digit-product sums of one chunk stay exact in FP32");

// digit pairs in order of level s + t, then s
__constant__ unsigned char kPairS[kPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2,
                                             3, 4, 5, 0, 1, 2, 3, 4, 5, 6, 0, 1, 2, 3, 4, 5, 6, 7};
__constant__ unsigned char kPairT[kPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3,
                                             2, 1, 0, 6, 5, 4, 3, 2, 1, 0, 7, 6, 5, 4, 3, 2, 1, 0};

__host__ __device__ inline int tiles_of(int d)
{
    const int nt = (d + kT - 1) / kT;
    return nt * (nt + 1) / 2;
}

// the job owning index `idx` of a launch and the index within the job (prefix[e]: first
// index of job e, prefix[E]: the total)
__device__ __forceinline__ int job_at(const unsigned* __restrict__ prefix, int E, unsigned idx, unsigned& local)
{
    int lo = 0, hi = E;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= idx) lo = mid; else hi = mid;
    }
    local = idx - prefix[lo];
    return lo;
}

// Column exponents e_j (|Xc_ij| < 2^e_j; 0 for a zero column) and zeroed sums. Block: 32
// columns x 32 row groups; the maximum of |Xc_ij| is taken on the bit patterns.
__global__ void __launch_bounds__(1024) k_cov_exp(const CovJob* __restrict__ jobs, const unsigned* __restrict__ prefix,
                                                  int E)
{
    unsigned lb;
    const CovJob& J = jobs[job_at(prefix, E, blockIdx.x, lb)];
    const int n = J.n, d = J.d;
    const int j = (int)lb * 32 + threadIdx.x;
    __shared__ unsigned long long sm[32][33];
    unsigned long long m = 0ull;
    if (j < d)
        for (int i = threadIdx.y; i < n; i += 32)
            m = max(m, (unsigned long long)__double_as_longlong(J.Xc[(size_t)i * d + j]) & 0x7FFFFFFFFFFFFFFFull);
    sm[threadIdx.y][threadIdx.x] = m;
    // the sums of columns j of this block (every row), zeroed before the tensor-core kernel adds into them
    if (j < d)
        for (int r = threadIdx.y; r < d; r += 32) J.acc[(size_t)r * d + j] = 0ll;
    __syncthreads();
    if (threadIdx.y == 0 && j < d) {
        for (int y = 1; y < 32; ++y) m = max(m, sm[y][threadIdx.x]);
        const int be = (int)(m >> 52);                 // biased exponent of the largest magnitude
        J.cexp[j] = m == 0ull ? 0 : (be == 0 ? -1022 : be - 1022);
    }
}

// 2^k for -1022 <= k <= 1023
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// Digit planes G[s][j][i] (BF16, dpad x npad per plane, zero padding) of the scaled, rounded
// columns. Block: a 32 x 32 tile (rows i, columns j), transposed through shared memory.
__global__ void __launch_bounds__(256) k_cov_digits(const CovJob* __restrict__ jobs,
                                                    const unsigned* __restrict__ prefix, int E)
{
    unsigned lb;
    const CovJob& J = jobs[job_at(prefix, E, blockIdx.x, lb)];
    const int n = J.n, d = J.d, npad = J.npad, dpad = J.dpad;
    const int ti = npad / 32;
    const int i0 = (int)(lb % ti) * 32, j0 = (int)(lb / ti) * 32;
    __shared__ __nv_bfloat16 t[kDig][32][33];
    const int j = j0 + threadIdx.x;
    const int e = j < d ? J.cexp[j] : 0;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = i0 + r;
        long long v = 0;
        if (i < n && j < d) {
            // Xc_ij 2^(55 - e_j) in two exact power-of-two steps (55 - e_j lies in [-970, 1077]; a
            // product that underflows is below 1/2 and rounds to 0 either way)
            const int a = (55 - e) / 2;
            v = __double2ll_rn(J.Xc[(size_t)i * d + j] * pow2(a) * pow2(55 - e - a));
        }
#pragma unroll
        for (int s = kDig - 1; s > 0; --s) {
            const long long g = ((v + 64) & 127) - 64;
            t[s][threadIdx.x][r] = __float2bfloat16_rn((float)g);
            v = (v - g) >> kDigBits;
        }
        t[0][threadIdx.x][r] = __float2bfloat16_rn((float)v);
    }
    __syncthreads();
    for (int s = 0; s < kDig; ++s)
        for (int c = threadIdx.y; c < 32; c += 8)
            J.G[((size_t)s * dpad + j0 + c) * npad + i0 + threadIdx.x] = t[s][c][threadIdx.x];
}

// What one work unit computes: acc[r][c] += sum_i A_r,i B_c,i over a 128 x 128 tile, the
// digit pairs of group grp. Rows of A come from plane set mapA (plane s: rows s planeA ..),
// rows of B from mapB; the output tile starts at (r0, c0) of the row-major int64 sums acc
// (leading dimension ld), rows < rows and columns < cols are kept, and with `upper` only
// elements with c >= r.
struct UnitView {
    const CUtensorMap* mapA;
    const CUtensorMap* mapB;
    int planeA, planeB, rowA0, rowB0, nkb, grp;
    long long* acc;
    int ld, rows, cols, r0, c0;
    bool upper;
    int* status;
};

// unit -> tile (jt <= kt) of the covariance and pair group
__device__ __forceinline__ void unit_tile(int d, unsigned local, int& jt, int& kt, int& grp)
{
    grp = (int)(local % kGroups);
    int l = (int)(local / kGroups);
    const int nt = (d + kT - 1) / kT;
    jt = 0;
    while (l >= nt - jt) {
        l -= nt - jt;
        ++jt;
    }
    kt = jt + l;
}

// the covariance: tiles on or above the diagonal of S, one plane set for both operands
struct CovUnits {
    const CovJob* jobs;
    const unsigned* prefix;
    int E;
    __device__ unsigned count() const { return prefix[E]; }
    __device__ UnitView operator()(unsigned u) const
    {
        unsigned local;
        const CovJob& J = jobs[job_at(prefix, E, u, local)];
        int jt, kt, grp;
        unit_tile(J.d, local, jt, kt, grp);
        return UnitView{J.gmap, J.gmap, J.dpad, J.dpad, jt * kT, kt * kT, J.npad / kKB, grp,
                        J.acc, J.d, J.d, J.d, jt * kT, kt * kT, true, J.status};
    }
};

// the forward substitution after kFwdBlock-column block b: rows i of the working Zc (plane set A)
// against rows 256 (b + 1) + j of L (plane set B), both over the block's 256 columns
struct FwdUnits {
    const FwdJob* jobs;
    const unsigned* prefix;
    int E, b;
    __device__ unsigned count() const { return prefix[E]; }
    __device__ UnitView operator()(unsigned u) const
    {
        unsigned local;
        const FwdJob& J = jobs[job_at(prefix, E, u, local)];
        const int c_first = kFwdBlock * (b + 1), rest = J.d - c_first;
        const int grp = (int)(local % kGroups), t = (int)(local / kGroups);
        const int nj = (rest + kT - 1) / kT;
        const int it = t / nj, jt = t % nj;
        return UnitView{J.mapA, J.mapB, J.npadA, J.dpadB, it * kT, jt * kT, kFwdBlock / kKB, grp,
                        J.acc + c_first, J.d, J.n, rest, it * kT, jt * kT, false, J.status};
    }
};

template <class Units>
__global__ void __launch_bounds__(kThreads, 1) k_digit_gemm(const Units units_of)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* full = bar;
    uint64_t* empty = full + kStages;
    uint64_t* acc_full = empty + kStages;
    uint64_t* acc_empty = acc_full + kAccBufs;
    uint64_t* mma_done = acc_empty + kAccBufs;
    uint32_t* sTmem = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* sAbort = reinterpret_cast<volatile int*>(sTmem + 1);
    int* sErr = const_cast<int*>(sAbort) + 1;  // CTA-local wait code (turned into the jobs' status)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned units = units_of.count();
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < kAccBufs; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kEpiWarps); }
        mbar_init(mma_done, 1);
        *sAbort = 0;
        *sErr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        tmem_alloc(sTmem, kAccBufs * kT);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *sTmem;

    if (warp == kTmaWarp) {
        if (lane == 0) {
            uint32_t si = 0;
            bool ok = true;
            for (unsigned u = blockIdx.x; u < units && ok; u += gridDim.x) {
                const UnitView v = units_of(u);
                for (int c0 = 0; c0 < v.nkb && ok; c0 += kChunkKB)
                    for (int p = v.grp * kPairsPerGroup; p < (v.grp + 1) * kPairsPerGroup && ok; ++p) {
                        const int ra = kPairS[p] * v.planeA + v.rowA0, rb = kPairT[p] * v.planeB + v.rowB0;
                        for (int kb = c0; kb < min(c0 + kChunkKB, v.nkb); ++kb, ++si) {
                            const int s = si % kStages;
                            if (!(ok = wait_bar(&empty[s], ((si / kStages) & 1u) ^ 1u, sAbort, sErr, 1))) break;
                            unsigned char* st = smem + s * kStageBytes;
                            mbar_arrive_expect_tx(&full[s], kStageBytes);
                            tma_load_2d(st, v.mapA, &full[s], kb * kKB, ra);
                            tma_load_2d(st + kTileBytes / 2, v.mapA, &full[s], kb * kKB, ra + 64);
                            tma_load_2d(st + kTileBytes, v.mapB, &full[s], kb * kKB, rb);
                            tma_load_2d(st + kTileBytes + kTileBytes / 2, v.mapB, &full[s], kb * kKB, rb + 64);
                        }
                    }
            }
            if (!ok) {
                // the copies this thread may still have in flight land before the CTA exits
                const uint32_t from = si > (uint32_t)kStages ? si - kStages : 0u;
                for (uint32_t i = from; i < si; ++i) {
                    const unsigned long long t0 = clock64();
                    while (!mbar_try_wait(&full[i % kStages], (i / kStages) & 1u) && clock64() - t0 < kWaitCycles) {}
                }
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            bool ok = true;
            uint32_t si = 0, ai = 0;
            const uint32_t idesc = idesc_bf16(kT, kT);
            for (unsigned u = blockIdx.x; u < units && ok; u += gridDim.x) {
                const UnitView v = units_of(u);
                for (int c0 = 0; c0 < v.nkb && ok; c0 += kChunkKB)
                    for (int q = 0; q < kPairsPerGroup && ok; ++q, ++ai) {
                        const int b = ai % kAccBufs;
                        if (!(ok = wait_bar(&acc_empty[b], ((ai / kAccBufs) & 1u) ^ 1u, sAbort, sErr, 2))) break;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem_base + (uint32_t)(b * kT);
                        for (int kb = c0; kb < min(c0 + kChunkKB, v.nkb); ++kb, ++si) {
                            const int s = si % kStages;
                            if (!(ok = wait_bar(&full[s], (si / kStages) & 1u, sAbort, sErr, 3))) break;
                            tc_fence_after();
                            const unsigned char* st = smem + s * kStageBytes;
                            const uint64_t adesc = sdesc_sw128(smem_u32(st));
                            const uint64_t bdesc = sdesc_sw128(smem_u32(st + kTileBytes));
#pragma unroll
                            for (int k = 0; k < kKB / 16; ++k)
                                umma_bf16(d_tmem, adesc + 2u * k, bdesc + 2u * k, idesc, (kb > c0 || k > 0) ? 1u : 0u);
                            umma_commit(&empty[s]);
                        }
                        if (ok) umma_commit(&acc_full[b]);
                    }
            }
            // every MMA this thread issued has finished before TMEM is released
            umma_commit(mma_done);
            const unsigned long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < kWaitCycles) {}
        }
    } else {
        // epilogue: row 32 (warp % 4) + lane of the tile, columns 32 (warp / 4) .. + 32
        const int row = 32 * (warp & 3) + lane, cq = 32 * (warp >> 2);
        const uint32_t lane_addr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16);
        uint32_t ai = 0;
        bool ok = true;
        for (unsigned u = blockIdx.x; u < units && ok; u += gridDim.x) {
            const UnitView v = units_of(u);
            // two's complement sums: the partial sums of the four pair groups may wrap, their total
            // (below 2^63 in magnitude) does not
            unsigned long long acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0ull;
            for (int ch = 0; ch < v.nkb && ok; ch += kChunkKB)
                for (int p = v.grp * kPairsPerGroup; p < (v.grp + 1) * kPairsPerGroup && ok; ++p, ++ai) {
                    const int b = ai % kAccBufs;
                    if (!(ok = wait_bar(&acc_full[b], (ai / kAccBufs) & 1u, sAbort, sErr, 4))) break;
                    tc_fence_after();
                    // P 2^(7 (14 - L) - 59) for level L = s + t: times 2^(39 - 7 L) for L <= 5,
                    // shifted right by 3 and 10 with rounding to nearest for L = 6 and 7
                    const int sh = 39 - kDigBits * (kPairS[p] + kPairT[p]);
                    const long long mul = sh >= 0 ? (1ll << sh) : 1ll;
                    const int rsh = sh >= 0 ? 0 : -sh;
                    const long long half = sh >= 0 ? 0ll : (1ll << (rsh - 1));
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t x[16];
                        tmem_ld16(lane_addr + (uint32_t)(b * kT + cq + 16 * h), x);
                        tmem_wait_ld();
                        if (h == 1) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[b]);
                        }
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            acc[16 * h + c] += (unsigned long long)(
                                ((long long)acc_to_int(__uint_as_float(x[c])) * mul + half) >> rsh);
                    }
                }
            if (!ok) break;
            // this unit's partial sums into the job's sums
            const int r = v.r0 + row;
            if (r < v.rows) {
                long long* dst = v.acc + (size_t)r * v.ld;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int col = v.c0 + cq + c;
                    if (col < v.cols && (!v.upper || col >= r))
                        atomicAdd(reinterpret_cast<unsigned long long*>(dst + col), acc[c]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    // after an expired wait every unit of this CTA may be incomplete: all their jobs fail
    if (*sErr != 0 && tid == 0)
        for (unsigned u = blockIdx.x; u < units; u += gridDim.x) atomicOr(units_of(u).status, kStatusTimeout);
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kAccBufs * kT);
    }
}

// S_jk = S_kj = sum_jk 2^(59 + e_j + e_k - 110) / (n - 1) from the sum of the element on or
// above the diagonal; one thread per element (j, k >= j) writes both halves.
__global__ void __launch_bounds__(256) k_cov_finish(const CovJob* __restrict__ jobs,
                                                    const unsigned* __restrict__ prefix, int E)
{
    unsigned lb;
    const CovJob& J = jobs[job_at(prefix, E, blockIdx.x, lb)];
    const int d = J.d;
    const size_t idx = (size_t)lb * 256 + threadIdx.x;
    if (idx >= (size_t)d * d) return;
    const int j = (int)(idx / d), k = (int)(idx % d);
    if (k < j) return;
    // the sum's scale 2^(59 + e_j + e_k - 110) in three exact power-of-two steps (each factor
    // normal and of sc's sign, so no partial product over- or underflows unless the result
    // does), then the denominator as a product with RN(1/(n - 1)): one rounding more than a
    // division
    const double x = __ll2double_rn(J.acc[idx]);
    const int sc = kShift - 110 + J.cexp[j] + J.cexp[k];
    const int a = sc / 3, b = (sc - a) / 2;
    const double v = __dmul_rn(__dmul_rn(__dmul_rn(x, pow2(a)), pow2(b)), pow2(sc - a - b)) * J.rinv;
    J.S[idx] = v;
    J.S[(size_t)k * d + j] = v;
}

// Digit planes after block b, one warp per row: rows [0, npadA) are rows of the working Zc
// over the block's columns [256 b, 256 b + 256) (zero past n), the next 128 ceil(rest / 128)
// rows are rows 256 (b + 1) + j of L over the same columns (zero past d). Each row's
// exponent (its largest magnitude below 2^e) as in k_cov_exp.
__global__ void __launch_bounds__(256) k_fwd_digits(const FwdJob* __restrict__ jobs,
                                                    const unsigned* __restrict__ prefix, int E, int b)
{
    unsigned lb;
    const FwdJob& J = jobs[job_at(prefix, E, blockIdx.x, lb)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c_first = kFwdBlock * (b + 1), rest = J.d - c_first;
    const int rowsB = (rest + kT - 1) / kT * kT;
    const int r = (int)lb * 8 + warp;
    if (r >= J.npadA + rowsB) return;
    const bool isA = r < J.npadA;
    const int rr = isA ? r : r - J.npadA;
    const bool valid = isA ? rr < J.n : rr < rest;
    const double* src = isA ? J.ZT + (size_t)rr * J.d + kFwdBlock * b : J.L + (size_t)(c_first + rr) * J.d + kFwdBlock * b;
    constexpr int kPer = kFwdBlock / 32;  // entries per lane
    double x[kPer];
    unsigned long long m = 0ull;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        x[q] = valid ? src[lane + 32 * q] : 0.0;
        m = max(m, (unsigned long long)__double_as_longlong(x[q]) & 0x7FFFFFFFFFFFFFFFull);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long o = ((unsigned long long)__shfl_xor_sync(0xffffffffu, (unsigned)(m >> 32), off) << 32) |
                                     (unsigned long long)__shfl_xor_sync(0xffffffffu, (unsigned)m, off);
        m = max(m, o);
    }
    const int be = (int)(m >> 52);
    const int e = m == 0ull ? 0 : (be == 0 ? -1022 : be - 1022);
    if (lane == 0 && valid) (isA ? J.expA : J.expB)[rr] = e;
    __nv_bfloat16* G = isA ? J.GA : J.GB;
    const size_t plane = (size_t)(isA ? J.npadA : J.dpadB) * kFwdBlock;
    const int a = (55 - e) / 2;
    const double s1 = pow2(a), s2 = pow2(55 - e - a);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        long long v = __double2ll_rn(x[q] * s1 * s2);
        __nv_bfloat16* g = G + (size_t)rr * kFwdBlock + lane + 32 * q;
#pragma unroll
        for (int sd = kDig - 1; sd > 0; --sd) {
            const long long dg = ((v + 64) & 127) - 64;
            g[sd * plane] = __float2bfloat16_rn((float)dg);
            v = (v - dg) >> kDigBits;
        }
        g[0] = __float2bfloat16_rn((float)v);
    }
}

// ZT_i,c -= sum_ic 2^(59 + e_i + e_c - 110) for the columns c past block b, each element
// rounded once; the sums are zeroed for the next block. One thread per element.
__global__ void __launch_bounds__(256) k_fwd_apply(const FwdJob* __restrict__ jobs, const unsigned* __restrict__ prefix,
                                                   int E, int b)
{
    unsigned lb;
    const FwdJob& J = jobs[job_at(prefix, E, blockIdx.x, lb)];
    const int c_first = kFwdBlock * (b + 1), rest = J.d - c_first;
    const size_t idx = (size_t)lb * 256 + threadIdx.x;
    if (idx >= (size_t)J.n * rest) return;
    const int i = (int)(idx / rest), j = (int)(idx % rest);
    const size_t at = (size_t)i * J.d + c_first + j;
    const double x = __ll2double_rn(J.acc[at]);
    J.acc[at] = 0ll;
    // the scale in three exact power-of-two steps (all of sc's sign, so no partial product over-
    // or underflows unless the result does)
    const int sc = kShift - 110 + J.expA[i] + J.expB[j];
    const int s1 = sc / 3, s2 = (sc - s1) / 2;
    J.ZT[at] = __dsub_rn(J.ZT[at], __dmul_rn(__dmul_rn(__dmul_rn(x, pow2(s1)), pow2(s2)), pow2(sc - s1 - s2)));
}

size_t cov_smem_bytes() { return 1024 + (size_t)kStages * kStageBytes + (2 * kStages + 2 * kAccBufs + 1) * 8 + 16; }

}  // namespace

int cov_tc_npad(int n) { return (n + kKB - 1) / kKB * kKB; }
int cov_tc_dpad(int d) { return (d + kT - 1) / kT * kT; }
size_t cov_tc_plane_bytes(int n, int d) { return (size_t)kDig * cov_tc_dpad(d) * cov_tc_npad(n) * 2; }
unsigned cov_tc_exp_blocks(int n, int d) { (void)n; return (unsigned)((d + 31) / 32); }
unsigned cov_tc_digit_blocks(int n, int d) { return (unsigned)(cov_tc_npad(n) / 32) * (unsigned)(cov_tc_dpad(d) / 32); }
unsigned cov_tc_units(int n, int d) { (void)n; return (unsigned)(tiles_of(d) * kGroups); }
unsigned cov_tc_finish_blocks(int n, int d) { (void)n; return (unsigned)(((size_t)d * d + 255) / 256); }

bool cov_tc_map(CUtensorMap* m, const __nv_bfloat16* G, int n, int d)
{
    return make_map_bf16(m, G, (uint64_t)cov_tc_npad(n), (uint64_t)kDig * cov_tc_dpad(d), kKB, 64);
}

cudaError_t cov_tc_launch(const CovJob* jobs, const unsigned* const prefix[4], const unsigned total[4], int E,
                          int device, int num_sms, cudaStream_t s)
{
    if (total[0]) k_cov_exp<<<total[0], dim3(32, 32), 0, s>>>(jobs, prefix[0], E);
    if (total[1]) k_cov_digits<<<total[1], dim3(32, 8), 0, s>>>(jobs, prefix[1], E);
    if (total[2]) {
        const size_t smem = cov_smem_bytes();
        const cudaError_t e = set_smem_limit(k_digit_gemm<CovUnits>, (int)smem, device);
        if (e != cudaSuccess) return e;
        const unsigned grid = std::min<unsigned>(total[2], (unsigned)num_sms);
        k_digit_gemm<CovUnits><<<grid, kThreads, smem, s>>>(CovUnits{jobs, prefix[2], E});
    }
    if (total[3]) k_cov_finish<<<total[3], 256, 0, s>>>(jobs, prefix[3], E);
    return cudaGetLastError();
}

cudaError_t prep_tc_setup(int device)
{
    const int smem = (int)cov_smem_bytes();
    cudaError_t e = set_smem_limit(k_digit_gemm<CovUnits>, smem, device);
    if (e == cudaSuccess) e = set_smem_limit(k_digit_gemm<FwdUnits>, smem, device);
    return e;
}

int fwd_tc_npadA(int n) { return (n + kT - 1) / kT * kT; }
int fwd_tc_dpadB(int d) { return d > kFwdBlock ? (d - kFwdBlock + kT - 1) / kT * kT : 0; }
size_t fwd_tc_plane_bytes_a(int n) { return (size_t)kDig * fwd_tc_npadA(n) * kFwdBlock * 2; }
size_t fwd_tc_plane_bytes_b(int d) { return (size_t)kDig * fwd_tc_dpadB(d) * kFwdBlock * 2; }

unsigned fwd_tc_digit_blocks(int n, int d, int b)
{
    const int rest = d - kFwdBlock * (b + 1);
    return rest > 0 ? (unsigned)((fwd_tc_npadA(n) + (rest + kT - 1) / kT * kT) / 8) : 0u;
}

unsigned fwd_tc_units(int n, int d, int b)
{
    const int rest = d - kFwdBlock * (b + 1);
    return rest > 0 ? (unsigned)(((n + kT - 1) / kT) * ((rest + kT - 1) / kT) * kGroups) : 0u;
}

unsigned fwd_tc_apply_blocks(int n, int d, int b)
{
    const int rest = d - kFwdBlock * (b + 1);
    return rest > 0 ? (unsigned)(((size_t)n * rest + 255) / 256) : 0u;
}

bool fwd_tc_maps(CUtensorMap* ma, CUtensorMap* mb, const FwdJob& j)
{
    return make_map_bf16(ma, j.GA, (uint64_t)kFwdBlock, (uint64_t)kDig * j.npadA, kKB, 64) &&
           make_map_bf16(mb, j.GB, (uint64_t)kFwdBlock, (uint64_t)kDig * j.dpadB, kKB, 64);
}

cudaError_t fwd_tc_launch(const FwdJob* jobs, const unsigned* const prefix[3], const unsigned total[3], int E, int b,
                          int device, int num_sms, cudaStream_t s)
{
    if (total[0]) k_fwd_digits<<<total[0], 256, 0, s>>>(jobs, prefix[0], E, b);
    if (total[1]) {
        const size_t smem = cov_smem_bytes();
        const cudaError_t e = set_smem_limit(k_digit_gemm<FwdUnits>, (int)smem, device);
        if (e != cudaSuccess) return e;
        const unsigned grid = std::min<unsigned>(total[1], (unsigned)num_sms);
        k_digit_gemm<FwdUnits><<<grid, kThreads, smem, s>>>(FwdUnits{jobs, prefix[1], E, b});
    }
    if (total[2]) k_fwd_apply<<<total[2], 256, 0, s>>>(jobs, prefix[2], E, b);
    return cudaGetLastError();
}

}  // namespace frr
