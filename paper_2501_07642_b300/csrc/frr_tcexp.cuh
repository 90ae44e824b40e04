// frr_tcexp.cuh -- descriptor of one experiment for the tensor-core balance kernel.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace frr {

// One experiment as the tensor kernel sees it (also the layout of the device table
// used by the batched launch). The tensor maps describe its Zc hi / lo arrays.
struct TcExp {
    CUtensorMap map_hi, map_lo;
    const uint64_t* binom;
    float* Mout;          // approximate M of draw first + i goes to Mout[i]
    uint64_t seed, first, B;
    uint32_t rk[20];      // Philox round keys of the seed (philox_round_keys)
    float c_M;
    int n, n1, d, kb, nkb, nchunks, exact;
    unsigned* hist0;      // NULL, or 4096 counters that also count bits [31:20] of each M_hat
    // failure-path test of the single-experiment launch only (zero otherwise): the covariate
    // tile producer issues nothing, and every bounded wait gives up after wait_cycles cycles
    int skip_tma;
    unsigned long long wait_cycles;
};

}  // namespace frr
