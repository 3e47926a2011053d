// deposit_comp.cu -- the warp-cooperative deposit kernels (coop.cuh) with compensated
// FP32 accumulation (precision PSE_FP32_COMPENSATED), in a translation unit of their own
// so that they compile in parallel with the FP64-reduction variants of deposit.cu.
#include "coop.cuh"

namespace pse {

cudaError_t launch_coop_comp(const DepositParams &p, bool stats, int blocks_per_sm, bool binned, int64_t max_items,
                             cudaStream_t st)
{
    return binned ? launch_coop<true, Acc::COMP>(p, stats, blocks_per_sm, max_items, st)
                  : launch_coop<false, Acc::COMP>(p, stats, blocks_per_sm, max_items, st);
}

}  // namespace pse
