// Direct-addressed strategy interface (pm_direct.cu).
#pragma once

#include "pm_common.cuh"
#include "pm_partition.cuh"

namespace pm {

struct DirectArgs {
    const u64 *A, *Ac;   // f: ranks (sorted), coefficients
    const u64 *B, *Bc;   // g
    const u32 *B32;      // low 32 bits of g's ranks (slot arithmetic is mod 2^32)
    u32 na, nb;
    const u64 *gb;       // G + 1 group boundaries (ranks)
    u32 ngroups;
    u64 lo;              // smallest product rank; group g writes from gb[g] - lo
    u32 *edges;          // scratch: 2 * na words per group
    u64 *okey, *ocoef;   // output scratch
    u64 *ucount;         // terms written per group
    Layout L;
};

size_t direct_smem_bytes(u32 slots, int kind);
u32 direct_max_slots(int kind);
u64 *direct_groups(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u64 lo, u64 end, u32 G,
                   u32 grid_l);
void launch_direct(Ctx &c, const DirectArgs &a, u32 slots, int kind);

}  // namespace pm
