// frr_gen.cuh -- regeneration of an assignment from its key, one warp per draw.
//
// Key-only storage (Sec. 2.1): an accepted draw is kept as (pool seed, draw
// index) and its assignment is rebuilt on demand. The mapping from key to
// assignment is this library's reading (the paper fixes no generator):
//   r_i  = word (i mod 4) of Philox4x32-10(counter = (i/4, 0, lo(b), hi(b)),
//                                           key = (lo(seed), hi(seed)))
//   unit i is treated iff (r_i, i) is among the n1 smallest pairs.
// Exact enumeration (Sec. 2.3) maps a colex rank to its n1-subset instead.
//
// Layout produced. Lane l of the warp owns Philox blocks j = 32k + l (k < KB),
// i.e. units 128k + 4l + c for c < 4. The treated flags are gathered with one
// warp ballot per (k, c), which yields 32-bit word m = 4k + c of the draw's
// bit row: bit l of word m is unit 128k + 4l + c. The GEMM K dimension uses
// this "K-order" (position p = 32m + l); the covariate rows are stored in the
// same order at init, so no permutation happens per draw.
#pragma once
#include <stdint.h>
#include <type_traits>

namespace frr {

constexpr uint32_t kFull = 0xffffffffu;

// Unit index held at K-order position p.
__host__ __device__ __forceinline__ int unit_of_kpos(int p)
{
    const int m = p >> 5, l = p & 31;
    return 128 * (m >> 2) + 4 * l + (m & 3);
}

// K-order position of unit i.
__host__ __device__ __forceinline__ int kpos_of_unit(int i)
{
    const int k = i >> 7, rem = i & 127, l = rem >> 2, c = rem & 3;
    return 32 * (4 * k + c) + l;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplier S-box, key bumped by the two Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a_lo = x0 * 0xD2511F53u;
        const uint32_t a_hi = __umulhi(x0, 0xD2511F53u);
        const uint32_t b_lo = x2 * 0xCD9E8D57u;
        const uint32_t b_hi = __umulhi(x2, 0xCD9E8D57u);
        const uint32_t y0 = b_hi ^ x1 ^ k0;
        const uint32_t y2 = a_hi ^ x3 ^ k1;
        x0 = y0;
        x1 = b_lo;
        x2 = y2;
        x3 = a_lo;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Round keys of Philox4x32-10 for a seed: rk[2 r], rk[2 r + 1] = (lo, hi of the seed) +
// r (0x9E3779B9, 0xBB67AE85), r < 10.
__host__ __device__ __forceinline__ void philox_round_keys(uint64_t seed, uint32_t (&rk)[20])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// The same rounds as philox4x32_10 with the round keys read from rk (kernel-parameter
// space when rk points there, so that the XORs take them as constant operands).
__device__ __forceinline__ void philox4x32_10_rk(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                                 const uint32_t* rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a_lo = x0 * 0xD2511F53u;
        const uint32_t a_hi = __umulhi(x0, 0xD2511F53u);
        const uint32_t b_lo = x2 * 0xCD9E8D57u;
        const uint32_t b_hi = __umulhi(x2, 0xCD9E8D57u);
        const uint32_t y0 = b_hi ^ x1 ^ rk[2 * round];
        const uint32_t y2 = a_hi ^ x3 ^ rk[2 * round + 1];
        x0 = y0;
        x1 = b_lo;
        x2 = y2;
        x3 = a_lo;
    }
}

// Words 4k .. 4k + 3 of a lane (units u .. u + 3 of Philox block k): the block's output,
// with units >= n set to 0xffffffff. Block k of the warp covers units 128k .. 128k + 127, so
// when all of them exist (a warp-uniform test) no per-word selects are issued (about nine
// integer instructions per block, on the pipe that generation keeps busiest).
template <int KB>
__device__ __forceinline__ void pad_block(uint32_t (&r)[4 * KB], int k, uint32_t x0, uint32_t x1, uint32_t x2,
                                          uint32_t x3, int u, int n)
{
    if (128 * (k + 1) <= n) {
        r[4 * k + 0] = x0;
        r[4 * k + 1] = x1;
        r[4 * k + 2] = x2;
        r[4 * k + 3] = x3;
    } else {
        r[4 * k + 0] = (u + 0 < n) ? x0 : 0xffffffffu;
        r[4 * k + 1] = (u + 1 < n) ? x1 : 0xffffffffu;
        r[4 * k + 2] = (u + 2 < n) ? x2 : 0xffffffffu;
        r[4 * k + 3] = (u + 3 < n) ? x3 : 0xffffffffu;
    }
}

template <int KB>
__device__ __forceinline__ void unit_words_rk(uint32_t (&r)[4 * KB], const uint32_t* rk, uint64_t draw, int n,
                                              int lane)
{
    const uint32_t d0 = (uint32_t)draw, d1 = (uint32_t)(draw >> 32);
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int j = 32 * k + lane;
        uint32_t x0 = (uint32_t)j, x1 = 0u, x2 = d0, x3 = d1;
        if (4 * j < n) philox4x32_10_rk(x0, x1, x2, x3, rk);
        pad_block<KB>(r, k, x0, x1, x2, x3, 4 * j, n);
    }
}

// The 4*KB unit words of this lane for draw `draw`; units >= n get 0xffffffff
// (they sort after every real unit because their index is larger).
template <int KB>
__device__ __forceinline__ void unit_words(uint32_t (&r)[4 * KB], uint64_t seed, uint64_t draw, int n, int lane)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t d0 = (uint32_t)draw, d1 = (uint32_t)(draw >> 32);
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int j = 32 * k + lane;
        uint32_t x0 = (uint32_t)j, x1 = 0u, x2 = d0, x3 = d1;
        if (4 * j < n) philox4x32_10(x0, x1, x2, x3, k0, k1);
        pad_block<KB>(r, k, x0, x1, x2, x3, 4 * j, n);
    }
}

template <int KB>
__device__ __forceinline__ int warp_count_le(const uint32_t (&r)[4 * KB], uint32_t t)
{
    // r <= t exactly when t - r does not borrow: the carry of each subtraction is
    // added to the count (two integer instructions per word)
    uint32_t c = 0;
#pragma unroll
    for (int e = 0; e < 4 * KB; ++e) {
        uint32_t scratch;
        asm("sub.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %1, 0;" : "=r"(scratch), "+r"(c) : "r"(t), "r"(r[e]));
    }
    return (int)__reduce_add_sync(kFull, c);
}

// Slot mask type: one bit per unit word held by the lane.
template <int KB>
using slot_mask_t = typename std::conditional<(4 * KB <= 32), uint32_t, uint64_t>::type;

// Treated flags (bit e = slot e = unit 128(e/4) + 4 lane + e%4) of the n1
// smallest (r, unit) pairs across the warp. Search for the n1-th smallest
// value v: interpolation on the empirical CDF (the words are uniform), with a
// bisection step whenever the bracket fails to halve; it stops early as soon as
// some t has exactly n1 words <= t. Each step strictly shrinks the bracket, so
// the loop ends after at most ~70 counts (about 5 on average at n = 1000). The
// interpolation only steers the search, so it is done in FP32.
// Outcome of the selection: normally a value t with exactly n1 words <= t (treated =
// r <= t); when the n1-th and (n1+1)-th words are equal, a per-slot mask instead.
template <int KB>
struct SelectOutcome {
    uint32_t t;
    bool tie;
    slot_mask_t<KB> mask;
};

template <int KB>
__device__ __forceinline__ SelectOutcome<KB> warp_select_smallest(const uint32_t (&r)[4 * KB], int n, int n1, int lane)
{
    using M = slot_mask_t<KB>;
    long long lo = -1, hi = 0xffffffffll;
    int clo = 0, chi = 128 * KB;
    // Only 32-bit integer <-> float conversions here: the 64-bit ones execute on the
    // (narrow) FP64 unit, which every generating warp would share.
    const float inv_n = __fdividef(1.0f, (float)n);
    long long t = (long long)__float2uint_rz(fminf((float)n1 * inv_n * 4294967296.0f, 4294967040.0f));
    const long long step = (long long)__float2uint_rz(4294967296.0f * inv_n);
    long long prev_span = hi - lo;
    bool bisect = false;
    for (int it = 0;; ++it) {
        const uint32_t tt = (uint32_t)t;
        const int c = warp_count_le<KB>(r, tt);
        if (c == n1) return SelectOutcome<KB>{tt, false, 0};
        if (c > n1) { hi = t; chi = c; } else { lo = t; clo = c; }
        const long long span = hi - lo;
        if (span <= 1) break;
        if (it == 0) {
            t += (long long)(n1 - c) * step + ((n1 > c) ? step / 2 : -step / 2);
        } else if (bisect) {
            t = lo + span / 2;
        } else {
            const float frac = __fdividef((float)(n1 - clo), (float)(chi - clo));
            const uint32_t span32 = span > 0xffffffffll ? 0xffffffffu : (uint32_t)span;
            t = lo + (long long)__float2uint_rz(__uint2float_rz(span32) * frac + 0.5f);
        }
        if (t <= lo) t = lo + 1;
        if (t >= hi) t = hi - 1;
        bisect = !bisect && (2 * span > prev_span);
        prev_span = span;
    }
    // Ties at v = hi: words < v are treated; of the words == v, the (n1 - clo)
    // with the smallest unit indices are treated. Unit order is k, then lane, then c.
    const uint32_t v = (uint32_t)hi;
    const int need = n1 - clo;
    M m = 0;
    int base = 0;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        int tl = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) tl += (r[4 * k + c] == v) ? 1 : 0;
        int incl = tl;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        int rank = base + incl - tl;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int e = 4 * k + c;
            if (r[e] < v) {
                m |= (M)1 << e;
            } else if (r[e] == v) {
                if (rank < need) m |= (M)1 << e;
                ++rank;
            }
        }
        base += __shfl_sync(kFull, incl, 31);
    }
    return SelectOutcome<KB>{0u, true, m};
}

// Writes the draw's bit row (4*KB words, K-order) to row[] (shared or global). Word e
// is the warp ballot of slot e; every lane stores the same value (one transaction).
template <int KB>
__device__ __forceinline__ void warp_store_bits(const SelectOutcome<KB>& sel, const uint32_t (&r)[4 * KB], uint32_t* row)
{
    constexpr int W = 4 * KB;
    if (!sel.tie) {
#pragma unroll
        for (int e = 0; e < W; ++e) row[e] = __ballot_sync(kFull, r[e] <= sel.t);
    } else {
#pragma unroll
        for (int e = 0; e < W; ++e) row[e] = __ballot_sync(kFull, (unsigned)((sel.mask >> e) & 1u));
    }
}

// Colex unranking (combinatorial number system): rank = sum_m C(c_m, m) with
// c_1 < ... < c_n1; returns the n-bit mask. binom[c * 64 + m] = C(c, m).
__device__ __forceinline__ uint64_t unrank_colex(uint64_t rank, int n, int n1, const uint64_t* binom)
{
    uint64_t mask = 0;
    int c = n - 1;
    for (int m = n1; m >= 1; --m) {
        while (binom[c * 64 + m] > rank) --c;
        mask |= 1ull << c;
        rank -= binom[c * 64 + m];
        --c;
    }
    return mask;
}

// Bit row (K-order) of an exact-enumeration mask; n <= 63 so every unit has k = 0
// and only words 0..3 can be non-zero.
__device__ __forceinline__ void warp_store_mask_bits(uint64_t mask, uint32_t* row, int lane, int words)
{
    uint32_t mine = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int u = 4 * lane + c;
        const unsigned bit = (u < 64) ? (unsigned)((mask >> u) & 1ull) : 0u;
        const uint32_t w = __ballot_sync(kFull, bit);
        if (lane == c) mine = w;
    }
    for (int q = lane; q < words; q += 32) row[q] = (q < 4) ? mine : 0u;
}

// Word c (c < 4) of the K-order bit row of an n <= 63 mask: bit l is unit 4l + c.
// The stride-4 bits are gathered by halving the gaps four times.
__device__ __forceinline__ uint32_t kword_of_mask(uint64_t mask, int c)
{
    uint64_t x = (mask >> c) & 0x1111111111111111ull;
    x = (x | (x >> 3)) & 0x0303030303030303ull;
    x = (x | (x >> 6)) & 0x000F000F000F000Full;
    x = (x | (x >> 12)) & 0x000000FF000000FFull;
    x = (x | (x >> 24)) & 0x000000000000FFFFull;
    return (uint32_t)x;
}

// Exact enumeration with one rank per lane (no warp collectives): the lane unranks its
// own colex rank and writes that draw's row (words 0..3 from the mask, the rest zero).
__device__ __forceinline__ void lane_exact_row(uint64_t rank, int n, int n1, const uint64_t* binom, uint32_t* row,
                                               int words)
{
    const uint64_t m = unrank_colex(rank, n, n1, binom);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (c < words) row[c] = kword_of_mask(m, c);
    for (int q = 4; q < words; ++q) row[q] = 0u;
}

// A Philox draw -> its bit row, with precomputed round keys (see unit_words_rk).
template <int KB>
__device__ __forceinline__ void warp_draw_bits_rk(const uint32_t* rk, uint64_t draw, int n, int n1, uint32_t* row,
                                                  int lane)
{
    uint32_t r[4 * KB];
    unit_words_rk<KB>(r, rk, draw, n, lane);
    warp_store_bits<KB>(warp_select_smallest<KB>(r, n, n1, lane), r, row);
}

// One draw -> its bit row. 4 * KB words are written.
template <int KB>
__device__ __forceinline__ void warp_draw_bits(bool exact, uint64_t seed, uint64_t draw, int n, int n1,
                                               const uint64_t* binom, uint32_t* row, int lane)
{
    if (exact) {
        uint64_t mask = 0;
        if (lane == 0) mask = unrank_colex(draw, n, n1, binom);
        mask = __shfl_sync(kFull, mask, 0);
        warp_store_mask_bits(mask, row, lane, 4 * KB);
    } else {
        uint32_t r[4 * KB];
        unit_words<KB>(r, seed, draw, n, lane);
        const SelectOutcome<KB> sel = warp_select_smallest<KB>(r, n, n1, lane);
        warp_store_bits<KB>(sel, r, row);
    }
}

}  // namespace frr
