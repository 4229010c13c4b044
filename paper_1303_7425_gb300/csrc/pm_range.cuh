// K-c/K-d interface (pm_range.cu).
#pragma once

#include "pm_common.cuh"

namespace pm {

struct RangeArgs {
    const u64 *fkey, *fcoef;  // sorted operand f: keys (sort) or ranks (direct), coefficients
    const u64 *gkey, *gcoef;  // sorted operand g
    u32 na, nb;
    const u64 *rlo, *rhi, *rO, *boff;  // ranges (pm_partition.cuh)
    u32 nranges;
    u64 *okey, *ocoef;  // output scratch: slot boff[k] onwards belongs to range k
    u64 *ucount;        // terms written per range
    Layout L;           // rank -> key conversion (direct)
    u32 *status;
};

size_t sort_smem_bytes(u32 chunk, int kind);
void launch_range_sort(Ctx &c, const RangeArgs &a, u32 chunk, int kind, unsigned grid);

}  // namespace pm
