// K-b/K-c/K-d, direct-addressed strategy (dense products).
//
// Work split: the output rank interval [lo, end) is cut into G groups at
// order statistics of the almost regular grid of Sec. 5 (each grid point
// gamma_{i,j} stands for the same number of term products, so equal numbers
// of sorted grid points per group give groups with about equal operation
// counts, as the paper's first step intends).  One CTA owns one group, so no
// two CTAs ever write the same output term (Alg. 1, second step).
//
// Inside a group the CTA slides a window [lo, hi) of at most `slots` ranks
// and keeps one shared-memory accumulator per rank.  For each window it
// needs, per row i of the pp-matrix, the first column with
// gamma_{i,j} >= lo and the first with gamma_{i,j} >= hi (FindEdge,
// Sec. 2).  Both edges move left as i grows, so each thread walks a
// contiguous chunk of rows as a staircase (O(n_a + n_b) per window for the
// whole CTA) after one binary search for its first row.
#include "pm_direct.cuh"

namespace pm {

constexpr int DT = 1024;          // threads per CTA
constexpr int DW = DT / 32;       // warps
constexpr int DROWS = DT;         // rows staged per pass

struct DTables {
    u32 *ra;    // (u32) rank of alpha_i
    u64 *ca;    // a_i
    u32 *jlo;   // first column in the window
    u32 *off;   // exclusive prefix of row spans (DROWS + 1)
};

constexpr size_t DTABLE_BYTES = (size_t)DROWS * (4 + 8 + 4) + (DROWS + 1) * 4 + 12;

__device__ __forceinline__ DTables carve_dtables(unsigned char *p)
{
    DTables t;
    t.ca = (u64 *)p;
    t.ra = (u32 *)(t.ca + DROWS);
    t.jlo = t.ra + DROWS;
    t.off = t.jlo + DROWS;
    return t;
}

// residue of a slot: 64-bit sum plus 8 per wrap of the sum
__device__ __forceinline__ u64 m61_slot(u64 sum, u32 nwraps)
{
    return m61_reduce(m61_reduce(sum) + 8ull * nwraps);
}

__device__ __forceinline__ u32 d_row_of(const u32 *off, u32 nrows, u32 p)
{
    u32 lo = 0, len = nrows;
    while (len > 0) {
        u32 half = len >> 1;
        if (off[lo + half] <= p) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo - 1;
}

// lower_bound(B, x) when it is known to be <= j: a short linear check, then a
// galloping search downwards (O(log of the distance moved))
__device__ __forceinline__ u32 walk_down(const u64 *__restrict__ B, u32 j, u64 x)
{
    if (j == 0 || __ldg(B + j - 1) < x) return j;
    u32 hi = j - 1;  // B[hi] >= x
    u32 step = 1, lo;
    for (;;) {
        if (hi < step) {
            lo = 0;
            break;
        }
        const u32 probe = hi - step;
        if (__ldg(B + probe) < x) {
            lo = probe + 1;
            break;
        }
        hi = probe;
        step <<= 1;
    }
    return lo + lower_bound_u64(B + lo, hi - lo, x);
}

// E0[i] = lower_bound(B, lo - A_i), E1[i] = lower_bound(B, hi - A_i) for rows
// i in [i0, i1); every such row has A_i + B_min < hi.  Returns the number of
// term products of this thread's rows inside [lo, hi).
__device__ __forceinline__ u64 staircase_edges(const u64 *__restrict__ A, const u64 *__restrict__ B, u32 nb,
                                               u32 i0, u32 i1, u64 lo, u64 hi, u32 *__restrict__ E0,
                                               u32 *__restrict__ E1)
{
    const u32 rows = i1 - i0;
    const u32 per = (rows + DT - 1) / DT;
    const u32 r0 = i0 + threadIdx.x * per;
    const u32 r1 = min(r0 + per, i1);
    if (r0 >= r1) return 0;
    u64 a = __ldg(A + r0);
    u32 j0 = lo > a ? lower_bound_u64(B, nb, lo - a) : 0u;
    u32 j1 = lower_bound_u64(B, nb, hi - a);
    E0[r0] = j0;
    E1[r0] = j1;
    u64 sum = j1 - j0;
    for (u32 i = r0 + 1; i < r1; i++) {
        a = __ldg(A + i);
        j0 = lo <= a ? 0u : walk_down(B, j0, lo - a);
        j1 = walk_down(B, j1, hi - a);
        E0[i] = j0;
        E1[i] = j1;
        sum += j1 - j0;
    }
    return sum;
}

template <int KIND>
__global__ void __launch_bounds__(DT, 1) k_direct(DirectArgs a, u32 slots)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 win[2];
    // M61: 64-bit sums [0, slots) then 32-bit wrap counts; I64: lo words
    // [0, slots) then hi words [slots, 2 slots)
    u64 *acc = (u64 *)smem;
    u32 *wraps = (u32 *)(acc + slots);
    DTables t = carve_dtables(smem + (size_t)slots * (KIND == PM_COEF_M61 ? 12 : 16));
    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const u32 g = blockIdx.x;
    if (g >= a.ngroups) return;
    const u64 glo = a.gb[g], ghi = a.gb[g + 1];
    u32 *E0 = a.edges + (size_t)g * 2 * a.na;
    u32 *E1 = E0 + a.na;
    const u64 bmin = __ldg(a.B), bmax = __ldg(a.B + a.nb - 1);
    const u64 obase = glo - a.lo;
    u64 run = 0;

    for (u64 lo = glo; lo < ghi;) {
        const u64 hi = ghi - lo > slots ? lo + slots : ghi;
        const u32 span = (u32)(hi - lo);
        if (tid == 0) {
            win[0] = lo > bmax ? lower_bound_u64(a.A, a.na, lo - bmax) : 0u;
            win[1] = lower_bound_u64(a.A, a.na, hi - bmin);
        }
        __syncthreads();
        const u32 i0 = win[0], i1 = win[1];
        u64 wprod = 0;
        if (i0 < i1) {
            u64 mine = staircase_edges(a.A, a.B, a.nb, i0, i1, lo, hi, E0, E1);
            block_exclusive_scan(mine, wprod, ws);  // also orders the edge writes before their reads
        }
        if (wprod == 0) {  // no term product lands in this window
            __syncthreads();  // every thread has read win[] before it is rewritten
            lo = hi;
            continue;
        }
        for (u32 s = tid; s < span; s += DT) {
            acc[s] = 0;
            if (KIND == PM_COEF_M61) wraps[s] = 0;
            else acc[slots + s] = 0;
        }
        __syncthreads();

        for (u32 base = i0; base < i1; base += DROWS) {
            const u32 i = base + tid;
            u64 len = 0;
            if (i < i1) {
                const u32 jl = E0[i], jh = E1[i];
                len = jh - jl;
                t.ra[tid] = (u32)__ldg(a.A + i);
                t.ca[tid] = __ldg(a.Ac + i);
                t.jlo[tid] = jl;
            }
            u64 total;
            const u64 ex = block_exclusive_scan(len, total, ws);
            t.off[tid] = (u32)ex;
            if (tid == 0) t.off[DROWS] = (u32)total;
            const u32 nrows = min(i1 - base, (u32)DROWS);
            __syncthreads();

            // warp w takes a contiguous slice of the pass's products; a lane
            // keeps its current row's data in registers
            const u32 tot = (u32)total;
            const u32 per_warp = ((tot + DW - 1) / DW + 31u) & ~31u;
            const u32 p0 = w * per_warp;
            const u32 p1 = min(p0 + per_warp, tot);
            u32 p = p0 + lane;
            if (p < p1) {
                u32 r = d_row_of(t.off, nrows, p);
                const u32 lo32 = (u32)lo;
                u32 rend = t.off[r + 1];
                u32 jbase = t.jlo[r] - t.off[r];
                u32 ra = t.ra[r] - lo32;
                u64 ca = t.ca[r];
                for (; p < p1; p += 32) {
                    if (p >= rend) {
                        do {
                            r++;
                        } while (t.off[r + 1] <= p);
                        rend = t.off[r + 1];
                        jbase = t.jlo[r] - t.off[r];
                        ra = t.ra[r] - lo32;
                        ca = t.ca[r];
                    }
                    const u32 j = jbase + p;
                    const u32 slot = ra + __ldg(a.B32 + j);
                    if (KIND == PM_COEF_M61) {
                        // 2^64 = 8 (mod p): count the 64-bit word's wraps
                        // beside it instead of repairing them in a loop
                        const u64 v = m61_mul_lazy(ca, __ldg(a.Bc + j));
                        const u64 old = atomicAdd(&acc[slot], v);
                        atomicAdd(&wraps[slot], (u32)(old + v < old));
                    } else {
                        u64 plo, phi;
                        mul_i64_wide((i64)ca, (i64)__ldg(a.Bc + j), plo, phi);
                        const u64 old = atomicAdd(&acc[slot], plo);
                        atomicAdd(&acc[slots + slot], phi + (old + plo < old ? 1ull : 0ull));
                    }
                }
            }
            __syncthreads();
        }

        // emit the window's non-zero slots in ascending order: warp w owns
        // the contiguous slots [w * chunk, (w + 1) * chunk); pass 1 counts,
        // one block scan places the warps, pass 2 writes
        const u32 chunk = ((span + DW - 1) / DW + 31u) & ~31u;
        const u32 s0 = w * chunk, s1 = min(s0 + chunk, span);
        u32 wcount = 0;
        for (u32 sb = s0; sb < s1; sb += 32) {
            const u32 s = sb + lane;
            bool nz = false;
            if (s < s1) nz = KIND == PM_COEF_M61 ? m61_slot(acc[s], wraps[s]) != 0 : (acc[s] | acc[slots + s]) != 0;
            wcount += __popc(__ballot_sync(0xffffffffu, nz));
        }
        u64 wtot;
        const u64 wbase = block_exclusive_scan(lane == 0 ? wcount : 0, wtot, ws);
        u64 put = obase + run + __shfl_sync(0xffffffffu, wbase, 0);
        for (u32 sb = s0; sb < s1; sb += 32) {
            const u32 s = sb + lane;
            u64 v0 = 0, v1 = 0;
            bool nz = false;
            if (s < s1) {
                if (KIND == PM_COEF_M61) {
                    v0 = m61_slot(acc[s], wraps[s]);
                    nz = v0 != 0;
                } else {
                    v0 = acc[s];
                    v1 = acc[slots + s];
                    nz = (v0 | v1) != 0;
                }
            }
            const u32 bal = __ballot_sync(0xffffffffu, nz);
            if (nz) {
                const u64 d = put + __popc(bal & ((1u << lane) - 1u));
                a.okey[d] = rank_to_key(a.L, lo + s);
                if (KIND == PM_COEF_M61) {
                    a.ocoef[d] = v0;
                } else {
                    a.ocoef[2 * d] = v0;
                    a.ocoef[2 * d + 1] = v1;
                }
            }
            put += __popc(bal);
        }
        run += wtot;
        __syncthreads();
        lo = hi;
    }
    if (tid == 0) a.ucount[g] = run;
}

// group boundaries at order statistics of the sorted grid sample
__global__ void k_group_bounds(const u64 *__restrict__ sample, u64 ns, u32 G, u64 lo, u64 end, u64 *__restrict__ gb)
{
    u32 m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > G) return;
    u64 v;
    if (m == 0) v = lo;
    else if (m == G) v = end;
    else v = sample[(u64)(((unsigned __int128)m * ns) / G)];
    gb[m] = v;
}

size_t direct_smem_bytes(u32 slots, int kind)
{
    return (size_t)slots * (kind == PM_COEF_M61 ? 12 : 16) + DTABLE_BYTES;
}

u32 direct_max_slots(int kind)
{
    // 227 KB of opt-in shared memory per CTA, minus tables and static use
    size_t avail = 227 * 1024 - DTABLE_BYTES - 512;
    return (u32)(avail / (kind == PM_COEF_M61 ? 12 : 16)) & ~1023u;
}

template <class K>
static void set_smem(K kernel, size_t bytes)
{
    PM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

u64 *direct_groups(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u64 lo, u64 end, u32 G,
                   u32 grid_l)
{
    u32 l = grid_l ? grid_l : 1;
    u32 si = na / l ? na / l : 1, sj = nb / l ? nb / l : 1;
    u32 stagger = (u32)(nb / (2ull * l));
    u32 R = (na + si - 1) / si, Cc = (nb + sj - 1) / sj;
    u64 total = (u64)R * Cc + Cc + R;
    u64 *cand = S.get<u64>(total);
    grid_sample(c, A, na, B, nb, si, sj, stagger, R, Cc, total, cand);
    radix_sort_pairs(c, S, cand, nullptr, nullptr, total, bit_length(end));
    u64 *gb = S.get<u64>(G + 1);
    k_group_bounds<<<(G + 256) / 256, 256, 0, c.s>>>(cand, total, G, lo, end, gb);
    PM_LAUNCHED(c);
    return gb;
}

void launch_direct(Ctx &c, const DirectArgs &a, u32 slots, int kind)
{
    size_t bytes = direct_smem_bytes(slots, kind);
    if (kind == PM_COEF_M61) {
        set_smem(k_direct<PM_COEF_M61>, bytes);
        k_direct<PM_COEF_M61><<<a.ngroups, DT, bytes, c.s>>>(a, slots);
    } else {
        set_smem(k_direct<PM_COEF_I64_ACC128>, bytes);
        k_direct<PM_COEF_I64_ACC128><<<a.ngroups, DT, bytes, c.s>>>(a, slots);
    }
    PM_LAUNCHED(c);
}

}  // namespace pm
