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
    u64 key_lo = 0, key_hi = ~0ull;  // only output keys in [key_lo, key_hi) (a slice of the product)
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

// The almost regular grid of Sec. 5 over the n_a x n_b pp-matrix for the
// parameter l (1-based i, j in the paper, 0-based here): rows i = 0, si,
// 2 si, ... with si = max(n_a / l, 1); in each, columns j = j0 + m sj with
// sj = max(n_b / l, 1) and j0 = stagger = n_b / (2 l) on every second grid
// row (the paper's alternating offset), else 0; then the last row (row
// n_a - 1 at columns m sj) and the last column (column n_b - 1 at rows
// m si).  Point p < R Cc is grid row p / Cc, column p % Cc; the next Cc
// points are the last row, the R after them the last column.  Columns past
// the matrix are clamped to its last column (duplicates are removed after
// the sort).
struct GridShape {
    u32 si, sj, stagger, R, Cc;
    u64 total;
};

__host__ __device__ inline GridShape grid_shape(u32 na, u32 nb, u32 l)
{
    GridShape g;
    if (l == 0) l = 1;
    g.si = na / l ? na / l : 1;
    g.sj = nb / l ? nb / l : 1;
    g.stagger = (u32)(nb / (2ull * l));
    g.R = (na + g.si - 1) / g.si;
    g.Cc = (nb + g.sj - 1) / g.sj;
    g.total = (u64)g.R * g.Cc + g.Cc + g.R;
    return g;
}

__device__ __forceinline__ void grid_point(const GridShape &g, u32 na, u32 nb, u64 p, u64 &i, u64 &j)
{
    const u64 interior = (u64)g.R * g.Cc;
    if (p < interior) {
        const u64 r = p / g.Cc, q = p % g.Cc;
        i = r * g.si;
        j = (r & 1) * g.stagger + q * g.sj;
    } else if (p < interior + g.Cc) {
        i = na - 1;
        j = (p - interior) * g.sj;
    } else {
        i = (p - interior - g.Cc) * g.si;
        j = nb - 1;
    }
    if (i > na - 1) i = na - 1;
    if (j > nb - 1) j = nb - 1;
}

// the grid's points A[i] + B[j]: g.total values into out
void grid_sample(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const GridShape &g, u64 *out);

// Step 1 of Alg. 1: the grid's points and gamma_end = A[na-1] + B[nb-1] + 1
// (exclusive end), sorted and deduplicated; *ns receives their number (one
// host read).  A and B: sorted keys (or ranks).
// With clamp_lo / clamp_hi, every splitter is first clamped into
// [clamp_lo, clamp_hi] (the splitters of a slice of the output key space).
u64 *grid_splitters(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u32 l, u64 end, u32 *ns,
                    u64 clamp_lo = 0, u64 clamp_hi = ~0ull);

// cnt[k] = #{(i, j) : A_i + B_j < Sp[k]} for the ns splitters (the
// cumulative operation counts of Alg. 2)
void count_below(Ctx &c, const u64 *A, u32 na, const u64 *B, u32 nb, const u64 *Sp, u32 ns, u64 *cnt);

// Alg. 2's split of intervals into nshards groups by cumulative operation
// count: cum[0..ns) ascending (cum[0] = 0, cum[ns-1] = the total), cut[m]
// (m = 0..nshards) the interval boundary index where shard m starts
// (cut[0] = 0, cut[nshards] = ns - 1): the first boundary whose count
// reaches m / nshards of the total, never before the previous cut.
void split_cumulative(const u64 *cum, u32 ns, u32 nshards, u32 *cut);

Ranges partition(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, const PartitionPlan &plan);

}  // namespace pm
