// K-c + K-d: the parallel step of Alg. 1.  One CTA owns one output range
// [lo, hi) at a time, so no other CTA ever touches its terms: the CTA
// (1) finds the rows of the pp-matrix that reach the range and, per row, the
//     first and one-past-last column inside it (FindEdge, Sec. 2: the
//     matrix is increasing along rows and columns, so each edge is a
//     lower-bound search on the sorted operand),
// (2) forms the range's term products, staging per-row data in shared memory
//     and reading the other operand's coefficients with coalesced loads,
// (3) accumulates them in shared memory -- the "MergeSort" of Alg. 1 -- with
//     a bucket sort of the range's (key, product) pairs on the top bits of
//     key - lo (radix sort where keys cluster), then a segmented reduction
//     (the direct-addressed strategy lives in pm_direct.cu),
// (4) writes its non-zero terms in ascending order to the range's slice of
//     the output scratch (concatenation happens in K-e).
#include "pm_blocksort.cuh"
#include "pm_range.cuh"

namespace pm {

constexpr int RK_THREADS = 512;
constexpr int RK_WARPS = RK_THREADS / 32;
constexpr int ROWS = RK_THREADS;  // rows staged per pass

// shared-memory row tables of one pass
struct RowTables {
    u64 *rkey;   // row key (or rank) alpha_i
    u64 *rcoef;  // a_i
    u32 *jlo;    // first column inside the range
    u32 *off;    // exclusive prefix of the row spans, ROWS + 1 entries
};

__device__ __forceinline__ RowTables carve_rows(unsigned char *p)
{
    RowTables t;
    t.rkey = (u64 *)p;
    t.rcoef = t.rkey + ROWS;
    t.jlo = (u32 *)(t.rcoef + ROWS);
    t.off = t.jlo + ROWS;
    return t;
}

constexpr size_t ROW_TABLE_BYTES = ROWS * (8 + 8 + 4) + (ROWS + 1) * 4 + 12;

// Stage rows [base, min(base + ROWS, i1)) and their column edges for the
// range [lo, hi); returns the number of term products of the pass.
__device__ __forceinline__ u32 stage_rows(const RangeArgs &a, const RowTables &t, u32 base, u32 i1, u64 lo, u64 hi,
                                          u64 *ws, u32 &nrows)
{
    const u32 tid = threadIdx.x;
    const u32 i = base + tid;
    u64 len = 0;
    if (i < i1) {
        u64 r = __ldg(a.fkey + i);
        u32 jl = lo > r ? lower_bound_u64(a.gkey, a.nb, lo - r) : 0u;
        u32 jh = lower_bound_u64(a.gkey, a.nb, hi - r);
        len = jh - jl;
        t.rkey[tid] = r;
        t.rcoef[tid] = __ldg(a.fcoef + i);
        t.jlo[tid] = jl;
    }
    u64 total;
    u64 ex = block_exclusive_scan(len, total, ws);
    t.off[tid] = (u32)ex;
    if (tid == 0) t.off[ROWS] = (u32)total;
    nrows = i1 - base < (u32)ROWS ? i1 - base : (u32)ROWS;
    __syncthreads();
    return (u32)total;
}

// rows of f that reach [lo, hi): alpha_i + beta_max >= lo and alpha_i + beta_min < hi
__device__ __forceinline__ void row_window(const RangeArgs &a, u64 lo, u64 hi, u32 &i0, u32 &i1)
{
    const u64 gmin = __ldg(a.gkey), gmax = __ldg(a.gkey + a.nb - 1);
    i0 = lo > gmax ? lower_bound_u64(a.fkey, a.na, lo - gmax) : 0u;
    i1 = lower_bound_u64(a.fkey, a.na, hi - gmin);
}

// row owning flattened product p: last r with off[r] <= p
__device__ __forceinline__ u32 row_of(const u32 *off, u32 nrows, u32 p)
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

// Visit the pass's products: warp w takes a contiguous slice, lanes stride
// by 32 inside it, so consecutive lanes read consecutive columns of g.
template <class F>
__device__ __forceinline__ void for_each_product(const RowTables &t, u32 nrows, u32 total, F &&fn)
{
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const u32 per_warp = ((total + RK_WARPS - 1) / RK_WARPS + 31u) & ~31u;
    const u32 p0 = w * per_warp;
    const u32 p1 = min(p0 + per_warp, total);
    u32 p = p0 + lane;
    if (p >= p1) return;
    u32 r = row_of(t.off, nrows, p);
    for (; p < p1; p += 32) {
        while (t.off[r + 1] <= p) r++;
        u32 j = t.jlo[r] + (p - t.off[r]);
        fn(r, j, p);
    }
}

// ---------------------------------------------------------------------------
// shared-memory radix sort + segmented reduction
// ---------------------------------------------------------------------------

constexpr int SORT_IPT_MAX = 8;  // chunk <= RK_THREADS * 8 = 4096

struct SortSmem {
    u64 *kA, *kB;     // keys relative to lo
    uint16_t *iA, *iB;  // product index
    u64 *cv;          // product coefficients (I64: lo[chunk], hi[chunk])
    u32 *hist;        // [RK_WARPS][256]
};

__device__ __forceinline__ SortSmem carve_sort(unsigned char *p, u32 chunk, int kind)
{
    SortSmem m;
    m.kA = (u64 *)p;
    m.kB = m.kA + chunk;
    m.cv = m.kB + chunk;
    u64 *after = m.cv + (size_t)chunk * (kind == PM_COEF_M61 ? 1 : 2);
    m.hist = (u32 *)after;
    m.iA = (uint16_t *)(m.hist + RK_WARPS * 256);
    m.iB = m.iA + chunk;
    return m;
}

template <int KIND>
__global__ void __launch_bounds__(RK_THREADS) k_range_sort(RangeArgs a, u32 chunk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 win[2];
    __shared__ u64 red[3 * RK_WARPS];
    constexpr bool W3 = KIND == PM_COEF_I64_ACC192;        // 192-bit sums
    constexpr u32 OW = KIND == PM_COEF_M61 ? 1 : (W3 ? 3 : 2);  // result words
    const size_t sort_bytes = (size_t)chunk * 8 * (KIND == PM_COEF_M61 ? 3 : 4) + RK_WARPS * 256 * 4 +
                              (size_t)chunk * 4;
    RowTables t = carve_rows(smem + ((sort_bytes + 15) & ~(size_t)15));
    const u32 tid = threadIdx.x;

    for (u32 k = blockIdx.x; k < a.nranges; k += gridDim.x) {
        const u64 lo = a.rlo[k], hi = a.rhi[k];
        const u64 O = a.rO[k];
        SortSmem m = carve_sort(smem, chunk, KIND);
        if (tid == 0) row_window(a, lo, hi, win[0], win[1]);
        __syncthreads();
        const u32 i0 = win[0], i1 = win[1];
        const u64 obase = a.boff[k];

        if (O > chunk) {
            // a single monomial with more products than the chunk: plain sum
            if (hi - lo != 1 && tid == 0) atomicOr(a.status, ST_INTERNAL);
            u64 s0 = 0, s1 = 0, s2 = 0;
            for (u32 base = i0; base < i1; base += ROWS) {
                u32 nrows;
                u32 total = stage_rows(a, t, base, i1, lo, hi, ws, nrows);
                for_each_product(t, nrows, total, [&](u32 r, u32 j, u32) {
                    if (KIND == PM_COEF_M61) {
                        s0 = m61_add(s0, m61_reduce(m61_mul_lazy(t.rcoef[r], __ldg(a.gcoef + j))));
                    } else {
                        u64 plo, phi;
                        mul_i64_wide((i64)t.rcoef[r], (i64)__ldg(a.gcoef + j), plo, phi);
                        if (W3) add192(s0, s1, s2, plo, phi);
                        else add128(s0, s1, plo, phi);
                    }
                });
                __syncthreads();
            }
            // block reduction of (s0, s1, s2)
            const u32 lane = tid & 31, w = tid >> 5;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                u64 o0 = __shfl_down_sync(0xffffffffu, s0, d), o1 = __shfl_down_sync(0xffffffffu, s1, d);
                u64 o2 = __shfl_down_sync(0xffffffffu, s2, d);
                if (KIND == PM_COEF_M61) s0 = m61_add(s0, o0);
                else if (W3) add192w(s0, s1, s2, o0, o1, o2);
                else add128(s0, s1, o0, o1);
            }
            if (lane == 0) {
                red[3 * w] = s0;
                red[3 * w + 1] = s1;
                red[3 * w + 2] = s2;
            }
            __syncthreads();
            if (tid == 0) {
                u64 r0 = 0, r1 = 0, r2 = 0;
                for (int ww = 0; ww < RK_WARPS; ww++) {
                    if (KIND == PM_COEF_M61) r0 = m61_add(r0, red[3 * ww]);
                    else if (W3) add192w(r0, r1, r2, red[3 * ww], red[3 * ww + 1], red[3 * ww + 2]);
                    else add128(r0, r1, red[3 * ww], red[3 * ww + 1]);
                }
                u64 cnt = 0;
                if ((r0 | r1 | r2) != 0) {
                    a.okey[obase] = lo;
                    a.ocoef[OW * obase] = r0;
                    if (OW > 1) a.ocoef[OW * obase + 1] = r1;
                    if (OW > 2) a.ocoef[OW * obase + 2] = r2;
                    cnt = 1;
                }
                a.ucount[k] = cnt;
            }
            __syncthreads();
            continue;
        }

        // (2) generate the range's products into shared memory
        u32 filled = 0;
        for (u32 base = i0; base < i1; base += ROWS) {
            u32 nrows;
            u32 total = stage_rows(a, t, base, i1, lo, hi, ws, nrows);
            const u32 at = filled;
            for_each_product(t, nrows, total, [&](u32 r, u32 j, u32 p) {
                const u32 q = at + p;
                if (q >= chunk) return;  // cannot happen when O_k <= chunk; keeps writes in bounds
                m.kA[q] = t.rkey[r] + __ldg(a.gkey + j) - lo;
                m.iA[q] = (uint16_t)q;
                if (KIND == PM_COEF_M61) {
                    m.cv[q] = m61_reduce(m61_mul_lazy(t.rcoef[r], __ldg(a.gcoef + j)));
                } else {
                    u64 plo, phi;
                    mul_i64_wide((i64)t.rcoef[r], (i64)__ldg(a.gcoef + j), plo, phi);
                    m.cv[q] = plo;
                    m.cv[chunk + q] = phi;
                }
            });
            filled += total;
            __syncthreads();
        }
        if (filled != O && tid == 0) atomicOr(a.status, ST_INTERNAL);
        const u32 n = filled < chunk ? filled : chunk;

        // (3) sort the keys (relative to lo, so inside [0, hi - 1 - lo]),
        // then reduce runs
        block_sort_interval<RK_THREADS, SORT_IPT_MAX>(m.kA, m.iA, m.kB, m.iB, n, 0, hi - 1 - lo, m.hist, ws);

        u64 run = 0;
        for (u32 c0 = 0; c0 < n; c0 += RK_THREADS) {
            const u32 i = c0 + tid;
            u64 v0 = 0, v1 = 0, v2 = 0;
            bool nz = false;
            if (i < n && (i == 0 || m.kA[i] != m.kA[i - 1])) {
                const u64 key = m.kA[i];
                for (u32 jj = i; jj < n && m.kA[jj] == key; jj++) {
                    const u32 src = m.iA[jj];
                    if (KIND == PM_COEF_M61) v0 = m61_add(v0, m.cv[src]);
                    else if (W3) add192(v0, v1, v2, m.cv[src], m.cv[chunk + src]);
                    else add128(v0, v1, m.cv[src], m.cv[chunk + src]);
                }
                nz = (v0 | v1 | v2) != 0;
            }
            u64 cnt;
            u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, ws);
            if (nz) {
                const u64 d = obase + run + pos;
                a.okey[d] = lo + m.kA[i];
                a.ocoef[OW * d] = v0;
                if (OW > 1) a.ocoef[OW * d + 1] = v1;
                if (OW > 2) a.ocoef[OW * d + 2] = v2;
            }
            run += cnt;
        }
        if (tid == 0) a.ucount[k] = run;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

size_t sort_smem_bytes(u32 chunk, int kind)
{
    size_t sort_bytes = (size_t)chunk * 8 * (kind == PM_COEF_M61 ? 3 : 4) + RK_WARPS * 256 * 4 + (size_t)chunk * 4;
    return ((sort_bytes + 15) & ~(size_t)15) + ROW_TABLE_BYTES;
}

template <class K>
static void set_smem(K kernel, size_t bytes)
{
    PM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

void launch_range_sort(Ctx &c, const RangeArgs &a, u32 chunk, int kind, unsigned grid)
{
    size_t bytes = sort_smem_bytes(chunk, kind);
    if (kind == PM_COEF_M61) {
        set_smem(k_range_sort<PM_COEF_M61>, bytes);
        k_range_sort<PM_COEF_M61><<<grid, RK_THREADS, bytes, c.s>>>(a, chunk);
    } else if (kind == PM_COEF_I64_ACC128) {
        set_smem(k_range_sort<PM_COEF_I64_ACC128>, bytes);
        k_range_sort<PM_COEF_I64_ACC128><<<grid, RK_THREADS, bytes, c.s>>>(a, chunk);
    } else {
        set_smem(k_range_sort<PM_COEF_I64_ACC192>, bytes);
        k_range_sort<PM_COEF_I64_ACC192><<<grid, RK_THREADS, bytes, c.s>>>(a, chunk);
    }
    PM_LAUNCHED(c);
}

}  // namespace pm
