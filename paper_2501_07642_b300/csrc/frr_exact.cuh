// frr_exact.cuh -- exact integer helpers of the tensor-core kernels whose FP32
// accumulators hold integers (the exact recheck, the covariance from digit products).
#pragma once
#include <cuda_runtime.h>

namespace frr {
namespace exact {

// Exact conversion of an integer-valued FP32 accumulator with |x| < 2^22: adding
// 1.5 * 2^23 places the integer in the low mantissa bits.
__device__ __forceinline__ int acc_to_int(float x) { return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000; }

// The signed 128-bit integer (hi, lo) times 2^-q as the nearest FP64 value (ties to even),
// built with integer instructions: normalise, keep 53 bits, round on the rest.
__device__ __forceinline__ double i128_to_double_scaled(long long hi, unsigned long long lo, int q)
{
    const bool neg = hi < 0;
    unsigned long long h = (unsigned long long)hi;
    if (neg) {
        lo = ~lo + 1ull;
        h = ~h + (lo == 0ull ? 1ull : 0ull);
    }
    if (h == 0ull && lo == 0ull) return 0.0;
    const int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)lo);
    if (lz >= 64) {
        h = lo << (lz - 64);
        lo = 0ull;
    } else if (lz > 0) {
        h = (h << lz) | (lo >> (64 - lz));
        lo <<= lz;
    }
    unsigned long long m = h >> 11;                 // 53 bits, the leading one at bit 52
    const bool round_bit = ((h >> 10) & 1ull) != 0ull;
    const bool sticky = (h & 0x3FFull) != 0ull || lo != 0ull;
    int e = 127 - lz;                               // value = m 2^(e - 52)
    if (round_bit && (sticky || (m & 1ull))) {
        ++m;
        if (m >> 53) {
            m >>= 1;
            ++e;
        }
    }
    const unsigned long long bits = ((unsigned long long)(e - q + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull) |
                                    (neg ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
}

}  // namespace exact
}  // namespace frr
