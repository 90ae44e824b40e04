// frr_balance_tc.cu -- split-BF16 tensor-core balance check (tcgen05 + TMA + TMEM).
#include "frr_internal.cuh"

namespace frr {

frr_status balance_tc_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout)
{
    (void)ctx; (void)seed; (void)exact; (void)first; (void)B; (void)Mout;
    return FRR_E_UNSUPPORTED;
}

}  // namespace frr
