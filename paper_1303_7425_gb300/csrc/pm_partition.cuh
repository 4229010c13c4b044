// K-b interface (pm_partition.cu).
#pragma once

#include "pm_common.cuh"

namespace pm {

struct PartitionPlan {
    u64 uniform_step = 0;   // > 0: start from a uniform split with this span (direct strategy)
    u32 grid_l = 0;         // otherwise: the Sec. 5 grid with this l
    u64 target = 0;         // split ranges with more term products than this
    bool hard_target = false;  // the target is a capacity (sort strategy), not a balance goal
    u64 max_split = 64;     // at most this many pieces per range per round
    u32 max_rounds = 64;
    u64 max_ranges = 1ull << 24;
};

// Non-empty output ranges [lo_k, hi_k), in ascending order.
struct Ranges {
    u32 n = 0;
    u64 *lo = nullptr, *hi = nullptr;
    u64 *O = nullptr;       // term products in the range
    u64 *boff = nullptr;    // exclusive scan of min(O_k, hi_k - lo_k): output slots
    u64 out_bound = 0;      // boff[n]
    u32 rounds = 0;
};

// the Sec. 5 grid points A[i] + B[j] (steps si, sj, alternate rows shifted by
// `stagger`, plus the last row and column): `total` values into out
void grid_sample(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, u32 si, u32 sj, u32 stagger, u32 R, u32 Cc,
                 u64 total, u64 *out);

Ranges partition(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, const PartitionPlan &plan);

}  // namespace pm
