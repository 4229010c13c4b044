// Direct-addressed strategy interface (pm_direct.cu).
#pragma once

#include "pm_common.cuh"
#include "pm_partition.cuh"

namespace pm {

struct DirectArgs {
    const u64 *A, *Ac;   // f: ranks (sorted), coefficients
    const u64 *B, *Bc;   // g
    const u32 *B32;      // low 32 bits of g's ranks (slot arithmetic is mod 2^32)
    const uint4 *Brec;   // ACC_L3: per column of g, {b_l, b_h, b_l + b_h, rank} (k_col_rec)
    const u32 *A32;      // f's ranks as u32 when the whole box fits in 32 bits, else null
    u32 na, nb;
    const u64 *gb;       // G + 1 group boundaries (ranks)
    u32 ngroups;
    u64 lo;              // smallest product rank; group g writes from gb[g] - lo
    const u64 *W;        // window boundaries; group g owns windows [wpos[g], wpos[g+1])
    const u64 *wpos;
    u32 *E;              // FindEdge table: E[b * na + i] for boundary b, row i
    u32 *i0s, *i1s;      // per boundary: first row reaching it, first row past it
    u64 *cnt;            // per boundary: term products with rank below it
    u64 *okey, *ocoef;   // output scratch
    u64 *ucount;         // terms written per window (set by launch_direct, nwin_max + 1 entries)
    Layout L;
    const u32 *abort;    // non-zero: a replayed plan's inputs no longer match it (may be null)
    u32 *order;          // windows, most expensive first (set by launch_direct)
    u32 *wnext;          // window counter of the persistent accumulate kernel
    u64 nwin_max;        // bound on the window count (host), slices for compaction
};

// hashed windows (sparse results in large rank boxes): the canonical
// operands and the product layout
struct HashInputs {
    const u64 *A, *Ac, *B, *Bc;  // ranks (sorted) and coefficients of f and g
    const u32 *B32;              // low 32 bits of g's ranks
    u32 na, nb;
    Layout L;
};
// h = f * g over the rank interval [lo, end) with hashed windows: several
// rounds (windows that overflow their table are split and run again), then
// the windows' terms are gathered in rank order into hkey/hcoef when the
// result fits `cap`.  Returns the result size; *rounds_out = rounds run,
// *windows_out += windows run over all rounds.
u64 hash_product(Ctx &c, Scratch &S, const HashInputs &in, int kind, int requested, u64 lo, u64 end, u64 products,
                 u64 *hkey, u64 *hcoef, u64 cap, u32 *rounds_out, u64 *windows_out);

size_t direct_smem_bytes(u32 slots, int kind, u64 min_n, int requested);
u32 direct_max_slots(int kind, u64 min_n, int requested);
// G + 1 group boundaries over [lo, end) with about equal cost; win: the
// window width (slots) the accumulate kernel will use; a group costs
// products + cost_row (rows staged) + cost_window (windows)
u64 *direct_groups(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u64 lo, u64 end, u32 G,
                   u32 grid_l, u64 products, u32 win, u32 cost_row, u32 cost_window, u64 nbk_max = 65536);
// Windows, FindEdge and the accumulate kernel.  On return a.W (window
// starts), a.ucount (terms per window) and a.nwin_max describe the result
// slices: window k's terms sit at a.W[k] - a.lo in the output scratch.
// ev_k0 / ev_k1 (may be null): events recorded around the accumulate launch
void launch_direct(Ctx &c, Scratch &S, DirectArgs &a, u32 slots, int kind, int requested, u64 end, u32 cost_row,
                   u32 cost_window, cudaEvent_t ev_k0 = nullptr, cudaEvent_t ev_k1 = nullptr);

}  // namespace pm
