// K-b/K-c/K-d, direct-addressed strategy (dense products).
//
// Work split: the output rank interval [lo, end) is cut into G groups with
// about equal cost.  Cost is sampled by the almost regular grid of Sec. 5
// (each grid point gamma_{i,j} stands for the same number of term products,
// as the paper's first step intends) plus each rank's share of the window
// costs (rows of f staged per window, fixed work per window); both go into
// a histogram over the interval, and the group boundaries sit where its
// cumulative cost crosses m / G of the total.
// One CTA owns one group, so no two CTAs ever write the same output term
// (Alg. 1, second step).
//
// Inside a group the CTA slides a window [lo, hi) of at most `slots` ranks
// and keeps one shared-memory accumulator per rank.  Each window needs, per
// row i of the pp-matrix, the first column with gamma_{i,j} >= lo and the
// first with gamma_{i,j} >= hi (FindEdge, Sec. 2); a separate kernel
// computes them for every window boundary beforehand (k_find_edge), so the
// accumulate kernel only reads them.
#include <algorithm>
#include <vector>

#include "pm_blocksort.cuh"
#include "pm_direct.cuh"

namespace pm {

constexpr int DT = 1024;          // threads per CTA
constexpr int DW = DT / 32;       // warps
constexpr int DRPT = 1;           // table rows per thread
constexpr int DROWS = DT * DRPT;  // rows staged per pass
constexpr int DCAND = 2;          // candidate rows looked at per thread and pass
static_assert(DCAND * DT < 4096, "kept-row count in 12 bits");

// shared-memory row tables of one pass: per staged row a 16-byte record
// (a_i as two words, rank of alpha_i minus the window start, first column
// minus the row's offset in the pass), so a lane that moves to the next row
// reloads its row state with one 16-byte load; plus the offsets
struct DTables {
    uint4 *rec;  // DROWS records
    u32 *off;    // exclusive prefix of row spans (DROWS + 1)
};

constexpr size_t DTABLE_BYTES = (size_t)DROWS * 16 + (DROWS + 1) * 4 + 12;

__device__ __forceinline__ DTables carve_dtables(unsigned char *p)
{
    DTables t;
    t.rec = (uint4 *)p;
    t.off = (u32 *)(t.rec + DROWS);
    return t;
}

// accumulator slots per window: as many as fit beside the tables, a
// multiple of 1024; a compile-time constant, so the accumulator's parallel
// arrays sit at fixed offsets from each other
constexpr u32 acc_stride(u32 bytes_per_slot)
{
    return (u32)((227 * 1024 - DTABLE_BYTES - 512) / bytes_per_slot) & ~1023u;
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

// first index in [0, n) with a[i] >= x (n if none); u32 or u64 keys, in
// shared or global memory
template <class K>
__device__ __forceinline__ u32 lower_bound_k(const K *a, u32 n, u64 x)
{
    u32 lo = 0, len = n;
    while (len > 0) {
        u32 half = len >> 1;
        if ((u64)a[lo + half] < x) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// lower_bound(B, x) when it is known to be <= j: a short linear check, then a
// galloping search downwards (O(log of the distance moved))
template <class K>
__device__ __forceinline__ u32 walk_down(const K *B, u32 j, u64 x)
{
    if (j == 0 || (u64)B[j - 1] < x) return j;
    u32 hi = j - 1;  // B[hi] >= x
    u32 step = 1, lo;
    for (;;) {
        if (hi < step) {
            lo = 0;
            break;
        }
        const u32 probe = hi - step;
        if ((u64)B[probe] < x) {
            lo = probe + 1;
            break;
        }
        hi = probe;
        step <<= 1;
    }
    return lo + lower_bound_k(B + lo, hi - lo, x);
}

// first index j' >= j with a[j'] >= x (n if none), a sorted: doubling steps
// from j, then a binary search of the last step
template <class K>
__device__ __forceinline__ u32 gallop_up_k(const K *a, u32 n, u32 j, u64 x)
{
    if (j >= n || (u64)a[j] >= x) return j;
    u32 lo = j, step = 1;  // a[lo] < x
    for (;;) {
        const u32 probe = lo + step;
        if (probe >= n || (u64)a[probe] >= x) {
            const u32 top = probe < n ? probe : n;
            return lo + 1 + lower_bound_k(a + lo + 1, top - lo - 1, x);
        }
        lo = probe;
        step <<= 1;
    }
}

// first index in [0, n) with a[i] >= x (n if none), by one warp: each round
// the 32 lanes probe 32 evenly spaced points of the interval that holds the
// answer, and the ballot of the probes below x narrows it 32-fold (three
// dependent loads for 32k elements instead of fifteen).  All lanes call.
template <class K>
__device__ __forceinline__ u32 warp_lower_bound(const K *__restrict__ a, u32 n, u64 x)
{
    const u32 lane = threadIdx.x & 31;
    u32 lo = 0, hi = n;  // the answer is in [lo, hi]
    while (lo < hi) {
        const u32 step = (hi - lo + 31) >> 5;
        const u32 probe = lo + (lane + 1) * step - 1;
        const bool below = probe < hi && (u64)a[probe] < x;
        const u32 k = (u32)__popc(__ballot_sync(0xffffffffu, below));  // a prefix of the lanes
        const u32 nhi = lo + (k + 1) * step - 1;
        lo += k * step;
        hi = nhi < hi ? nhi : hi;
    }
    return lo;
}

// FindEdge (Sec. 2) for the window boundaries: for boundary x = W[b] and
// every row i that reaches it, E[b][i] = #{j : beta_j < x - alpha_i}.  Rows
// below i0 (alpha_i + beta_max < x) have all n_b columns below x, rows from
// i1 on (alpha_i + beta_min >= x) none; cnt[b] = #{(i, j) : gamma_ij < x}.
// The row edges move left as i grows, so each thread walks a contiguous
// chunk of rows as a staircase after one binary search; g's keys are
// staged in shared memory when they fit, and so are the row edges, which
// then go out with coalesced stores (a thread's chunk of rows would give
// each lane a different line).  Warps 0 and 1 find i0 and i1 while the
// others stage g.  The grid is sized by an upper bound on the boundaries;
// blocks past their count return at once.
template <class K>
__global__ void __launch_bounds__(DT) k_find_edge(const K *__restrict__ A, const K *__restrict__ B, u32 na, u32 nb,
                                                  const u64 *__restrict__ W, const u64 *__restrict__ nbound_minus1,
                                                  u32 *__restrict__ E, u32 *__restrict__ i0s,
                                                  u32 *__restrict__ i1s, u64 *__restrict__ cnt, u32 stage,
                                                  u32 stage_e)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 rows[2];
    const u64 nbound = *nbound_minus1 + 1;
    if (blockIdx.x >= nbound) return;
    K *Bs = (K *)smem;
    u32 *Es = (u32 *)(smem + (stage ? ((size_t)nb * sizeof(K) + 15) / 16 * 16 : 0));
    const u64 bmin = (u64)B[0], bmax = (u64)B[nb - 1];
    const u32 w = threadIdx.x >> 5;
    for (u64 b = blockIdx.x; b < nbound; b += gridDim.x) {
        const u64 x = W[b];
        if (w == 0) {
            const u32 r = x > bmax ? warp_lower_bound(A, na, x - bmax) : 0u;
            if (threadIdx.x == 0) rows[0] = r;
        } else if (w == 1) {
            const u32 r = x > bmin ? warp_lower_bound(A, na, x - bmin) : 0u;
            if (threadIdx.x == 32) rows[1] = r;
        } else if (stage && b == blockIdx.x) {
            for (u32 j = threadIdx.x - 64; j < nb; j += DT - 64) Bs[j] = B[j];
        }
        __syncthreads();
        const K *Bp = stage ? Bs : B;
        const u32 i0 = rows[0], i1 = rows[1];
        u32 *Eb = E + b * na;
        u32 *Ew = stage_e ? Es : Eb;  // row i at Ew[i - eo]: Es holds rows [i0, i1)
        const u32 eo = stage_e ? i0 : 0u;
        u64 sum = 0;
        const u32 per = (i1 - i0 + DT - 1) / DT;
        const u32 r0 = i0 + threadIdx.x * per;
        const u32 r1 = min(r0 + per, i1);
        if (r0 < r1) {
            u32 j = lower_bound_k(Bp, nb, x - (u64)A[r0]);
            Ew[r0 - eo] = j;
            sum = j;
            for (u32 i = r0 + 1; i < r1; i++) {
                j = walk_down(Bp, j, x - (u64)A[i]);
                Ew[i - eo] = j;
                sum += j;
            }
        }
        u64 total;
        block_exclusive_scan(sum, total, ws);  // its barriers publish Es
        if (stage_e)
            for (u32 i = i0 + threadIdx.x; i < i1; i += DT) Eb[i] = Es[i - i0];
        if (threadIdx.x == 0) {
            cnt[b] = total + (u64)i0 * nb;
            i0s[b] = i0;
            i1s[b] = i1;
        }
        __syncthreads();
    }
}

// windows of at most `slots` ranks inside each group
__global__ void k_window_count(const u64 *__restrict__ gb, u32 G, u32 slots, u64 *__restrict__ nw)
{
    u32 g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const u64 span = gb[g + 1] - gb[g];
    nw[g] = (span + slots - 1) / slots;
}

__global__ void k_window_bounds(const u64 *__restrict__ gb, u32 G, u32 slots, const u64 *__restrict__ wpos,
                                u64 *__restrict__ W)
{
    u32 g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    for (u64 k = 0, n = wpos[g + 1] - wpos[g]; k < n; k++) W[wpos[g] + k] = gb[g] + k * slots;
    if (g == G - 1) W[wpos[G]] = gb[G];
}

// One product stream of a lane: flattened index p in [p, end) of the pass,
// with its row's data cached in registers.
struct Stream {
    u32 p, end, r, rend, jbase, ra;
    u64 ca;
};

// The same for the column-record path (ACC_L3): the row's coefficient
// halves and their sum, and a pointer to the column record of product p
// that moves with p (the pass's end is kept by the caller).
struct StreamR {
    u32 p, r, rend, ra, al, ah, sa;
    const uint4 *col;
};

__device__ __forceinline__ void stream_load_row(Stream &c, const DTables &t)
{
    const uint4 q = t.rec[c.r];
    c.ca = (u64)q.x | ((u64)q.y << 32);
    c.ra = q.z;
    c.jbase = q.w;
    c.rend = t.off[c.r + 1];
}

__device__ __forceinline__ void streamr_load_row(StreamR &c, const DTables &t, const uint4 *brec)
{
    const uint4 q = t.rec[c.r];
    c.al = q.x;
    c.ah = q.y;
    c.sa = q.x + q.y;
    c.ra = q.z;
    c.col = brec + (u32)(q.w + c.p);
    c.rend = t.off[c.r + 1];
}

__device__ __forceinline__ void streamr_init(StreamR &c, const DTables &t, u32 nrows, u32 p, u32 end,
                                             const uint4 *brec)
{
    c.p = p;
    if (p < end) {
        c.r = d_row_of(t.off, nrows, p);
        streamr_load_row(c, t, brec);
    }
}

__device__ __forceinline__ void streamr_advance_row(StreamR &c, const DTables &t, const uint4 *brec)
{
    if (c.p >= c.rend) {
        do {
            c.r++;
        } while (t.off[c.r + 1] <= c.p);
        streamr_load_row(c, t, brec);
    }
}

__device__ __forceinline__ void stream_init(Stream &c, const DTables &t, u32 nrows, u32 p, u32 end)
{
    c.p = p;
    c.end = end;
    if (p < end) {
        c.r = d_row_of(t.off, nrows, p);
        stream_load_row(c, t);
    }
}

__device__ __forceinline__ void stream_advance_row(Stream &c, const DTables &t)
{
    if (c.p >= c.rend) {
        do {
            c.r++;
        } while (t.off[c.r + 1] <= c.p);
        stream_load_row(c, t);
    }
}

// ---------------------------------------------------------------------------
// shared-memory accumulators, one slot per rank of the window
//   ACC_W64: mod p; a 64-bit sum and a 32-bit count of its wraps
//            (2^64 = 8 mod p), 12 bytes per slot;
//   ACC_L16: mod p; the lazily reduced product (< 2^62) split into four
//            16-bit limbs, each added into its own 32-bit counter with a
//            fire-and-forget reduction (one bank word each, no return
//            value); exact while a slot receives at most 65537 products,
//            i.e. when min(n_f, n_g) <= 65537 (one product per row and
//            per column at most), 16 bytes per slot;
//   ACC_I128: int64 inputs; 128-bit sum as lo and hi words, 16 bytes;
//   ACC_I192: int64 inputs; 192-bit sum in three words, each word's atomic
//            add returning the carry into the next, 24 bytes.
// ---------------------------------------------------------------------------
//   ACC_L3:  mod p, direct kernel only; the product (< 2^64) split into
//            limbs of 22, 21 and 21 bits, each added into its own 32-bit
//            counter with a fire-and-forget reduction, 12 bytes per slot.
//            A slot receives at most one product per row, and a pass of
//            the direct kernel stages at most L3_ROWS = 1023 rows; between
//            passes every slot is normalised (its value mod p split back
//            into the three limbs, the first below 2^22), so a counter
//            never exceeds (1 + 1023)(2^22 - 1) < 2^32.  One reduction per
//            product fewer than ACC_L16, and 4/3 as many slots per window.
enum { ACC_W64 = 0, ACC_L16 = 1, ACC_I128 = 2, ACC_I192 = 3, ACC_L3 = 4 };
constexpr u32 L3_ROWS = DROWS - 1;

template <int ACC, u32 STRIDE = 0>
struct Acc {
    static constexpr u32 bytes = (ACC == ACC_W64 || ACC == ACC_L3) ? 12 : (ACC == ACC_I192 ? 24 : 16);
    static constexpr u32 words = ACC == ACC_I192 ? 3 : (ACC == ACC_I128 ? 2 : 1);  // result words
    // array stride (a window may use fewer slots)
    static constexpr u32 slots = STRIDE ? STRIDE : acc_stride(bytes);
    u64 *w;      // ACC_W64: sums; ACC_I128/I192: word k of slot s at w[k * slots + s]
    u32 *c;      // ACC_W64: wrap counts; ACC_L16, ACC_L3: limb counters, limb k at [k * slots, (k+1) * slots)

    __device__ __forceinline__ void carve(unsigned char *p)
    {
        w = (u64 *)p;
        c = ACC == ACC_W64 ? (u32 *)(w + slots) : (u32 *)p;
    }
    __device__ __forceinline__ void zero(u32 s)
    {
        if (ACC == ACC_W64) {
            w[s] = 0;
            c[s] = 0;
        } else if (ACC == ACC_L16) {
            c[s] = 0;
            c[slots + s] = 0;
            c[2 * slots + s] = 0;
            c[3 * slots + s] = 0;
        } else if (ACC == ACC_L3) {
            c[s] = 0;
            c[slots + s] = 0;
            c[2 * slots + s] = 0;
        } else {
            w[s] = 0;
            w[slots + s] = 0;
            if (ACC == ACC_I192) w[2 * slots + s] = 0;
        }
    }
    // the product of a row coefficient and a column coefficient: for the
    // mod-p accumulators both come split (m61_split_row / m61_split_col)
    // and the product is m61_mul_split's (< 2^64; the limbs and the wrap
    // count take any 64-bit value); the integer kinds take them as they are
    __device__ __forceinline__ void add_split(u32 s, u64 a, u64 b)
    {
        if (ACC == ACC_W64) {
            const u64 v = m61_mul_split(a, b);
            const u64 old = atomicAdd(&w[s], v);
            atomicAdd(&c[s], (u32)(old + v < old));
        } else if (ACC == ACC_L16) {
            const u64 v = m61_mul_split(a, b);
            atomicAdd(&c[s], (u32)v & 0xFFFFu);
            atomicAdd(&c[slots + s], (u32)(v >> 16) & 0xFFFFu);
            atomicAdd(&c[2 * slots + s], (u32)(v >> 32) & 0xFFFFu);
            atomicAdd(&c[3 * slots + s], (u32)(v >> 48));
        } else if (ACC == ACC_L3) {
            add_l3(s, m61_mul_split(a, b));
        } else {
            add(s, a, b);
        }
    }
    __device__ __forceinline__ void add_l3(u32 s, u64 v)
    {
        atomicAdd(&c[s], (u32)v & 0x3FFFFFu);
        atomicAdd(&c[slots + s], (u32)(v >> 22) & 0x1FFFFFu);
        atomicAdd(&c[2 * slots + s], (u32)(v >> 43));
    }
    // the value of three limb counters c0 + c1 2^22 + c2 2^43 (each < 2^32)
    // mod p: c2 2^43 = (c2 >> 21) 2^64 + (c2 & (2^21 - 1)) 2^43 and
    // 2^64 = 8 (mod p)
    static __device__ __forceinline__ u64 l3_value(u32 c0, u32 c1, u32 c2)
    {
        const u64 x = (u64)c0 + ((u64)c1 << 22) + 8ull * (c2 >> 21);  // < 2^55
        const u64 y = (u64)(c2 & 0x1FFFFFu) << 43;                    // < 2^64
        return m61_add(m61_reduce(x), m61_reduce(y));
    }
    // ACC_L3 between passes: the slot's value mod p back in the three limbs
    __device__ __forceinline__ void normalize(u32 s)
    {
        if (ACC != ACC_L3) return;
        const u32 c0 = c[s], c1 = c[slots + s], c2 = c[2 * slots + s];
        if ((c0 | c1 | c2) == 0) return;
        const u64 v = l3_value(c0, c1, c2);
        c[s] = (u32)v & 0x3FFFFFu;
        c[slots + s] = (u32)(v >> 22) & 0x1FFFFFu;
        c[2 * slots + s] = (u32)(v >> 43);
    }
    __device__ __forceinline__ void add(u32 s, u64 a, u64 b)
    {
        if (ACC == ACC_W64) {
            const u64 v = m61_mul_lazy(a, b);
            const u64 old = atomicAdd(&w[s], v);
            atomicAdd(&c[s], (u32)(old + v < old));
        } else if (ACC == ACC_L16) {
            const u64 v = m61_mul_lazy(a, b);
            atomicAdd(&c[s], (u32)v & 0xFFFFu);
            atomicAdd(&c[slots + s], (u32)(v >> 16) & 0xFFFFu);
            atomicAdd(&c[2 * slots + s], (u32)(v >> 32) & 0xFFFFu);
            atomicAdd(&c[3 * slots + s], (u32)(v >> 48));
        } else if (ACC == ACC_L3) {
            add_l3(s, m61_mul_lazy(a, b));
        } else if (ACC == ACC_I128) {
            u64 plo, phi;
            mul_i64_wide((i64)a, (i64)b, plo, phi);
            const u64 old = atomicAdd(&w[s], plo);
            atomicAdd(&w[slots + s], phi + (old + plo < old ? 1ull : 0ull));
        } else {
            // the product sign-extended to 192 bits, word by word; each
            // atomic add's carry (from the value it returns) goes to the
            // next word, so the three words hold the exact sum
            u64 plo, phi;
            mul_i64_wide((i64)a, (i64)b, plo, phi);
            const u64 ext = (u64)((i64)phi >> 63);
            const u64 o0 = atomicAdd(&w[s], plo);
            const u64 t = phi + (o0 + plo < o0 ? 1ull : 0ull);
            const u64 c1a = t < phi ? 1ull : 0ull;
            const u64 o1 = atomicAdd(&w[slots + s], t);
            const u64 c1b = o1 + t < o1 ? 1ull : 0ull;
            atomicAdd(&w[2 * slots + s], ext + c1a + c1b);
        }
    }
    // emission, first pass: the slot's value (a residue mod p in v0, or the
    // two's complement words v0, v1, v2), left in the slot in a form take()
    // reads back with fewer loads: a residue as two 32-bit words in the
    // first two arrays (ACC_L16) or as the whole sum (ACC_W64)
    __device__ __forceinline__ bool finalize(u32 s, u64 &v0, u64 &v1, u64 &v2)
    {
        const bool nz = value(s, v0, v1, v2);
        if (ACC == ACC_W64) {
            w[s] = v0;
            c[s] = 0;
        } else if (ACC == ACC_L16) {
            c[s] = (u32)v0;
            c[slots + s] = (u32)(v0 >> 32);
            c[2 * slots + s] = 0;
            c[3 * slots + s] = 0;
        } else if (ACC == ACC_L3) {
            c[s] = (u32)v0;
            c[slots + s] = (u32)(v0 >> 32);
            c[2 * slots + s] = 0;
        }
        return nz;
    }
    // emission, second pass: the value finalize() left, and the slot cleared
    // for the next window
    __device__ __forceinline__ void take(u32 s, u64 &v0, u64 &v1, u64 &v2)
    {
        v1 = 0;
        v2 = 0;
        if (ACC == ACC_W64) {
            v0 = w[s];
            w[s] = 0;
        } else if (ACC == ACC_L16 || ACC == ACC_L3) {
            v0 = (u64)c[s] | ((u64)c[slots + s] << 32);
            c[s] = 0;
            c[slots + s] = 0;
        } else {
            v0 = w[s];
            v1 = w[slots + s];
            w[s] = 0;
            w[slots + s] = 0;
            if (ACC == ACC_I192) {
                v2 = w[2 * slots + s];
                w[2 * slots + s] = 0;
            }
        }
    }
    // the slot's value: residue mod p (v1 = v2 = 0), or the integer's words
    __device__ __forceinline__ bool value(u32 s, u64 &v0, u64 &v1, u64 &v2) const
    {
        v1 = 0;
        v2 = 0;
        if (ACC == ACC_W64) {
            v0 = m61_reduce(m61_reduce(w[s]) + 8ull * c[s]);
            return v0 != 0;
        } else if (ACC == ACC_L16) {
            // sum = L0 + L1 2^16 + L2 2^32 + L3 2^48 with L_k < 2^32
            const u64 l0 = c[s], l1 = c[slots + s], l2 = c[2 * slots + s], l3 = c[3 * slots + s];
            u64 lo = l0 + (l1 << 16);               // < 2^49
            u64 hi = 0;
            add128(lo, hi, l2 << 32, l2 >> 32);
            add128(lo, hi, l3 << 48, l3 >> 16);
            // 2^64 = 8 (mod p); hi < 2^17
            v0 = m61_reduce(m61_reduce(lo) + 8ull * hi);
            return v0 != 0;
        } else if (ACC == ACC_L3) {
            v0 = l3_value(c[s], c[slots + s], c[2 * slots + s]);
            return v0 != 0;
        } else {
            v0 = w[s];
            v1 = w[slots + s];
            if (ACC == ACC_I192) v2 = w[2 * slots + s];
            return (v0 | v1 | v2) != 0;
        }
    }
};

template <int ACC>
__global__ void __launch_bounds__(DT, 1) k_direct(DirectArgs a, u32 slots)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    Acc<ACC> acc;
    acc.carve(smem);
    DTables t = carve_dtables(smem + (size_t)Acc<ACC>::slots * Acc<ACC>::bytes);
    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ u32 s_next, s_cand;
    // inputs that no longer match a replayed plan could put products
    // outside the windows; such a replay computes nothing (the window
    // counts stay zero)
    if (a.abort && *a.abort) return;
    const u32 nb = a.nb, na = a.na;
    const u64 nwin = a.wpos[a.ngroups];
    // every slot starts at zero; each window's emission clears the slots
    // it read, so the next window starts from zero again
    for (u32 x = tid; x < Acc<ACC>::slots; x += DT) acc.zero(x);

    // persistent: take windows from a device counter, most expensive first
    // (the order k_window_order wrote), so the cheap ones fill the tail
    for (;;) {
        if (tid == 0) s_next = atomicAdd(a.wnext, 1u);
        __syncthreads();
        const u32 wk = s_next;
        __syncthreads();
        if (wk >= nwin) break;
        const u64 bw = a.order[wk];
        const u64 lo = a.W[bw], hi = a.W[bw + 1];
        const u32 span = (u32)(hi - lo);
        if (a.cnt[bw + 1] == a.cnt[bw]) continue;  // no term product lands in this window
        // rows reaching the window: [i0(lo), i1(hi)); edges below i1(lo) and
        // from i0(hi) on are stored, the others are 0 and n_b
        const u32 i0 = a.i0s[bw], i1 = a.i1s[bw + 1];
        const u32 i1lo = a.i1s[bw], i0hi = a.i0s[bw + 1];
        const u32 *Elo = a.E + bw * na, *Ehi = Elo + na;
        __syncthreads();

        // passes: each stages up to DROWS rows that have products in the
        // window (about half of the rows reaching it by their bounds have
        // none), taken in row order from the next DCAND * DT candidates
        for (u32 cand = i0; cand < i1;) {
            // thread tid looks at candidates cand + tid * DCAND + [0, DCAND);
            // one scan counts the kept rows (low 12 bits) and their products
            // (high bits); the records need the rows' offsets, so they are
            // written after it
            u32 lens[DCAND], jls[DCAND], ras[DCAND];
            u64 cas[DCAND];
            u64 packed = 0;
#pragma unroll
            for (int k = 0; k < DCAND; k++) {
                const u32 i = cand + tid * DCAND + k;
                lens[k] = 0;
                jls[k] = 0;
                ras[k] = 0;
                cas[k] = 0;
                if (i < i1) {
                    jls[k] = i < i1lo ? Elo[i] : 0u;
                    const u32 jh = i >= i0hi ? Ehi[i] : nb;
                    lens[k] = jh - jls[k];
                }
                if (lens[k]) {
                    ras[k] = (u32)__ldg(a.A + i) - (u32)lo;
                    cas[k] = __ldg(a.Ac + i);
                    if (ACC == ACC_W64 || ACC == ACC_L16 || ACC == ACC_L3) cas[k] = m61_split_row(cas[k]);
                    packed += ((u64)lens[k] << 12) | 1u;
                }
            }
            u64 ptot;
            const u64 ex = block_exclusive_scan(packed, ptot, ws);
            // rows per pass: the table's size, one fewer for ACC_L3 (its
            // counters' bound between normalisations)
            constexpr u32 RMAX = ACC == ACC_L3 ? L3_ROWS : (u32)DROWS;
            const u32 kept_all = (u32)(ptot & 4095u);
            const bool cut = kept_all > RMAX;
            u32 kept = (u32)(ex & 4095u);
            u32 off = (u32)(ex >> 12);
#pragma unroll
            for (int k = 0; k < DCAND; k++) {
                if (lens[k]) {
                    const u32 i = cand + tid * DCAND + k;
                    if (kept < RMAX) {
                        t.off[kept] = off;
                        t.rec[kept] = make_uint4((u32)cas[k], (u32)(cas[k] >> 32), ras[k], jls[k] - off);
                        off += lens[k];
                    } else if (kept == RMAX) {
                        // the first row that does not fit starts the next pass
                        t.off[RMAX] = off;
                        s_cand = i;
                    }
                    kept++;
                }
            }
            if (!cut && tid == 0) t.off[kept_all] = (u32)(ptot >> 12);
            __syncthreads();
            const u32 nrows = cut ? RMAX : kept_all;
            const u32 next = cut ? s_cand : cand + DCAND * DT;

            // warp w takes a contiguous slice of the pass's products; each
            // lane runs two independent streams over its two halves so the
            // loads and multiplies of one overlap the latency of the other
            const u32 tot = t.off[nrows];
            const u32 per_warp = ((tot + DW - 1) / DW + 63u) & ~63u;
            const u32 p0 = w * per_warp;
            const u32 p1 = min(p0 + per_warp, tot);
            const u32 pm = min(p0 + per_warp / 2, p1);
            if constexpr (ACC == ACC_L3) {
                // one 16-byte column record per product, through a pointer
                // that moves with the product index; the product by three
                // multiplies (m61_mul_k3)
                StreamR sa, sb;
                streamr_init(sa, t, nrows, p0 + lane, pm, a.Brec);
                streamr_init(sb, t, nrows, pm + lane, p1, a.Brec);
                while (sa.p < pm || sb.p < p1) {
                    const bool va = sa.p < pm, vb = sb.p < p1;
                    uint4 qa = make_uint4(0, 0, 0, 0), qb = make_uint4(0, 0, 0, 0);
                    if (va) {
                        streamr_advance_row(sa, t, a.Brec);
                        qa = __ldg(sa.col);
                    }
                    if (vb) {
                        streamr_advance_row(sb, t, a.Brec);
                        qb = __ldg(sb.col);
                    }
                    if (va) acc.add_l3(sa.ra + qa.w, m61_mul_k3(sa.al, sa.ah, sa.sa, qa.x, qa.y, qa.z));
                    if (vb) acc.add_l3(sb.ra + qb.w, m61_mul_k3(sb.al, sb.ah, sb.sa, qb.x, qb.y, qb.z));
                    sa.p += 32;
                    sb.p += 32;
                    sa.col += 32;
                    sb.col += 32;
                }
            } else {
            Stream sa, sb;
            stream_init(sa, t, nrows, p0 + lane, pm);
            stream_init(sb, t, nrows, pm + lane, p1);
            while (sa.p < sa.end || sb.p < sb.end) {
                const bool va = sa.p < sa.end, vb = sb.p < sb.end;
                u32 ja = 0, jb = 0, ba = 0, bb = 0;
                u64 ga = 0, gbv = 0;
                if (va) {
                    stream_advance_row(sa, t);
                    ja = sa.jbase + sa.p;
                    ba = __ldg(a.B32 + ja);
                    ga = __ldg(a.Bc + ja);
                }
                if (vb) {
                    stream_advance_row(sb, t);
                    jb = sb.jbase + sb.p;
                    bb = __ldg(a.B32 + jb);
                    gbv = __ldg(a.Bc + jb);
                }
                if (va) acc.add_split(sa.ra + ba, sa.ca, ga);
                if (vb) acc.add_split(sb.ra + bb, sb.ca, gbv);
                sa.p += 32;
                sb.p += 32;
            }
            }
            __syncthreads();
            if (ACC == ACC_L3 && next < i1) {
                // another pass follows: bring every counter back below its
                // limb's width
                for (u32 x = tid; x < span; x += DT) acc.normalize(x);
                __syncthreads();
            }
            cand = next;
        }

        // emit the window's non-zero slots in ascending order: warp w owns
        // the contiguous slots [w * chunk, (w + 1) * chunk); pass 1 computes
        // the values and counts, one block scan places the warps, pass 2
        // writes and clears the slots (warp-private, so no barrier between)
        const u32 chunk = ((span + DW - 1) / DW + 31u) & ~31u;
        const u32 s0 = w * chunk, s1 = min(s0 + chunk, span);
        u32 wcount = 0;
        for (u32 sb = s0; sb < s1; sb += 32) {
            const u32 s = sb + lane;
            bool nz = false;
            u64 x0, x1, x2;
            if (s < s1) nz = acc.finalize(s, x0, x1, x2);
            wcount += __popc(__ballot_sync(0xffffffffu, nz));
        }
        u64 wtot;
        const u64 wbase = block_exclusive_scan(lane == 0 ? wcount : 0, wtot, ws);
        // the window's terms go to its own part of the scratch, at its
        // first rank; compaction concatenates the windows in rank order
        u64 put = (lo - a.lo) + __shfl_sync(0xffffffffu, wbase, 0);
        for (u32 sb = s0; sb < s1; sb += 32) {
            const u32 s = sb + lane;
            u64 v0 = 0, v1 = 0, v2 = 0;
            if (s < s1) acc.take(s, v0, v1, v2);
            const bool nz = (v0 | v1 | v2) != 0;
            const u32 bal = __ballot_sync(0xffffffffu, nz);
            if (nz) {
                const u64 d = put + __popc(bal & ((1u << lane) - 1u));
                a.okey[d] = rank_to_key(a.L, lo + s);
                constexpr u32 W = Acc<ACC>::words;
                a.ocoef[W * d] = v0;
                if (W > 1) a.ocoef[W * d + 1] = v1;
                if (W > 2) a.ocoef[W * d + 2] = v2;
            }
            put += __popc(bal);
        }
        if (tid == 0) a.ucount[bw] = wtot;
        __syncthreads();
    }
}

// g's coefficients (residues mod p) in the split form of m61_mul_split
__global__ void k_split_col(const u64 *__restrict__ b, u64 *__restrict__ out, u32 n)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = m61_split_col(b[i]);
}

// g's columns as 16-byte records for m61_mul_k3: the coefficient's 31-bit
// halves, their sum, and the rank's low 32 bits
__global__ void k_col_rec(const u64 *__restrict__ b, const u32 *__restrict__ r32, uint4 *__restrict__ out, u32 n)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u64 v = b[i];
    const u32 bl = (u32)(v & 0x7FFFFFFFull), bh = (u32)(v >> 31);
    out[i] = make_uint4(bl, bh, bl + bh, r32[i]);
}

// Order of the windows for the persistent accumulate kernel: descending
// estimated cost (term products + cost_row rows staged + cost_window), by
// 64 power-of-two classes -- largest-first scheduling needs no more than an
// approximate order.  One CTA; windows at and past the device's window count
// are not listed.
__global__ void __launch_bounds__(1024) k_window_order(const u64 *__restrict__ cnt, const u32 *__restrict__ i0s,
                                                       const u32 *__restrict__ i1s, const u64 *__restrict__ nwin_p,
                                                       u64 cost_row, u64 cost_window, u32 *__restrict__ order)
{
    __shared__ u32 hist[64];
    __shared__ u32 base[64];
    const u64 nwin = *nwin_p;
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    auto cls = [&](u64 b) {
        const u64 prod = cnt[b + 1] - cnt[b];
        const u64 rows = i1s[b + 1] > i0s[b] ? i1s[b + 1] - i0s[b] : 0;
        const u64 cost = prod ? prod + cost_row * rows + cost_window : 0;
        return cost ? 63u - (u32)(63 - __clzll((long long)cost)) : 63u;  // 0 = most expensive
    };
    for (u64 b = threadIdx.x; b < nwin; b += blockDim.x) atomicAdd(&hist[cls(b)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 run = 0;
        for (int k = 0; k < 64; k++) {
            base[k] = run;
            run += hist[k];
        }
    }
    __syncthreads();
    for (u64 b = threadIdx.x; b < nwin; b += blockDim.x) order[atomicAdd(&base[cls(b)], 1u)] = (u32)b;
}

// Weighted histogram of the cost samples over NBK buckets of [lo, end):
// every grid point of Sec. 5 (steps si, sj, alternate rows shifted by
// `stagger`, plus the last row and column) adds wg to its bucket.
__global__ void k_grid_hist(const u64 *__restrict__ A, u32 na, const u64 *__restrict__ B, u32 nb, GridShape g,
                            u64 lo, u64 bw, u64 nbk, u64 wg, u64 *__restrict__ hist)
{
    const u64 p = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.total) return;
    u64 i, j;
    grid_point(g, na, nb, p, i, j);
    u64 k = (A[i] + B[j] - lo) / bw;
    if (k >= nbk) k = nbk - 1;
    atomicAdd(&hist[k], wg);
}

// Every bucket also carries its share of the window costs.  A window of
// `win` ranks starting at the bucket looks at the rows of f whose products
// can land in it -- alpha_i in [x - beta_max, x + win - beta_min) -- and the
// accumulate kernel's time per group measures as about
//     products + cost_row (rows reaching its windows) + cost_window (windows)
// in units of one term product (per-group timings of the dense workloads;
// since the passes stage only rows with products, 3 and 23000 by default;
// the autotuner picks the weights per shape class).  K_b = cost_row rows + cost_window is
// a window's cost near bucket b; a bucket of bw ranks carries bw / win of
// it (kw keeps K_b for the refinement below).
// (Both histogram kernels run HB-thread blocks, one bucket per thread, and
// leave the sum of each block's final bucket values in part[block] for
// k_group_cut.)
constexpr int HB = 256;

// sum over the block of one value per thread, in thread 0; all threads call
__device__ __forceinline__ u64 block_sum_u64(u64 v, u64 *ws)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    u64 s = 0;
    if (threadIdx.x == 0)
        for (u32 q = 0; q < (blockDim.x >> 5); q++) s += ws[q];
    return s;
}

__global__ void __launch_bounds__(HB) k_hist_rows(const u64 *__restrict__ A, u32 na, const u64 *__restrict__ B,
                                                  u32 nb, u64 lo, u64 bw, u64 win, u64 nbk, u64 cost_row,
                                                  u64 cost_window, u64 *__restrict__ hist, u64 *__restrict__ kw,
                                                  u64 *__restrict__ part)
{
    __shared__ u64 ws[32];
    const u64 k = (u64)blockIdx.x * HB + threadIdx.x;
    u64 h = 0;
    if (k < nbk) {
        const u64 bmin = B[0], bmax = B[nb - 1];
        const u64 x0 = lo + k * bw, x1 = x0 + win;
        const u32 i_lo = x0 > bmax ? lower_bound_u64(A, na, x0 - bmax) : 0u;
        const u32 i_hi = x1 > bmin ? lower_bound_u64(A, na, x1 - bmin) : 0u;
        const u64 rows = i_hi > i_lo ? i_hi - i_lo : 0;
        const u64 K = cost_row * rows + cost_window;
        kw[k] = K;
        h = hist[k] + (u64)(((unsigned __int128)K * bw) / win) + 1;
        hist[k] = h;
    }
    const u64 t = block_sum_u64(h, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// A group narrower than a window still pays one whole window, which the
// per-bucket share above charged only span / win of: its buckets get the
// rest, K_b bw (1 / span - 1 / win), before the groups are cut again.
__global__ void __launch_bounds__(HB) k_hist_narrow(const u64 *__restrict__ gb, u32 G, u64 lo, u64 bw, u64 win,
                                                    u64 nbk, const u64 *__restrict__ kw, u64 *__restrict__ hist,
                                                    u64 *__restrict__ part)
{
    __shared__ u64 ws[32];
    const u64 k = (u64)blockIdx.x * HB + threadIdx.x;
    u64 h = 0;
    if (k < nbk) {
        h = hist[k];
        const u64 x0 = lo + k * bw;
        // the group holding x0: last g with gb[g] <= x0
        u32 a = 0, n = G;
        while (n > 1) {
            const u32 hh = n >> 1;
            if (gb[a + hh] <= x0) {
                a += hh;
                n -= hh;
            } else {
                n = hh;
            }
        }
        const u64 span = gb[a + 1] - gb[a];
        if (span != 0 && span < win) {
            h += (u64)(((unsigned __int128)kw[k] * bw * (win - span)) / ((unsigned __int128)span * win));
            hist[k] = h;
        }
    }
    const u64 t = block_sum_u64(h, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Group boundaries from the bucket costs: with c_i the cost of the buckets
// below i (c_0 = 0, c_nbk = W), group m (0 < m < G) starts at bucket
// i(m) = the first i with c_i >= t_m = floor(W m / G), i.e. at lo + i(m) bw
// (at most end); gb[0] = lo and gb[G] = end.  One pass: block b takes
// GC_BUCKETS consecutive buckets [K0, K1), finds c_K0 from the histogram
// kernels' per-block sums, scans its buckets into shared memory, and owns
// the groups whose target falls in (c_K0, c_K1] (block 0 also those with
// t_m = 0): two divisions per block give their range of m, one per group
// its target, and a binary search over the block's scanned costs its
// bucket.
constexpr int GC_T = 256, GC_PER = 4;
constexpr u32 GC_BUCKETS = GC_T * GC_PER;
static_assert(GC_BUCKETS % HB == 0, "whole histogram blocks per cut block");

// floor((x y + a) / z) without overflow of x y + a; 64-bit arithmetic when
// it cannot overflow (a 128-bit division is a long software routine)
__device__ __forceinline__ u64 muldiv_floor(u64 x, u64 y, u64 a, u64 z)
{
    if (y == 0 || x <= (~0ull - a) / y) return (x * y + a) / z;
    return (u64)(((unsigned __int128)x * y + a) / z);
}

__global__ void __launch_bounds__(GC_T) k_group_cut(const u64 *__restrict__ hist, const u64 *__restrict__ part,
                                                    u32 nparts, u64 nbk, u32 G, u64 lo, u64 end, u64 bw,
                                                    u64 *__restrict__ gb)
{
    __shared__ u64 ws[32];
    __shared__ u64 cs[GC_BUCKETS + 1];  // cs[j] = c_{K0 + j}
    const u32 tid = threadIdx.x;
    const u64 K0 = (u64)blockIdx.x * GC_BUCKETS;
    const u32 nloc = (u32)(nbk - K0 < GC_BUCKETS ? nbk - K0 : GC_BUCKETS);
    const u32 pb = blockIdx.x * (GC_BUCKETS / HB);  // histogram blocks before this block's buckets
    // the cost below the block and the total, reduced together (one
    // barrier), while the block's own buckets load
    __shared__ u64 red[2][GC_T / 32];
    u64 below = 0, all = 0;
    for (u32 q = tid; q < nparts; q += GC_T) {
        const u64 v = part[q];
        all += v;
        if (q < pb) below += v;
    }
    u64 h[GC_PER];
    u64 mine = 0;
#pragma unroll
    for (int t = 0; t < GC_PER; t++) {
        const u32 j = tid * GC_PER + t;
        h[t] = j < nloc ? hist[K0 + j] : 0;
        mine += h[t];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        all += __shfl_xor_sync(0xffffffffu, all, d);
        below += __shfl_xor_sync(0xffffffffu, below, d);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = all;
        red[1][tid >> 5] = below;
    }
    __syncthreads();
    u64 W = 0, base = 0;
#pragma unroll
    for (int q = 0; q < GC_T / 32; q++) {
        W += red[0][q];
        base += red[1][q];
    }
    u64 tot;
    u64 c = base + block_exclusive_scan(mine, tot, ws);
#pragma unroll
    for (int t = 0; t < GC_PER; t++) {
        const u32 j = tid * GC_PER + t;
        if (j < nloc) cs[j] = c;
        c += h[t];
    }
    if (tid == 0) cs[nloc] = base + tot;
    if (blockIdx.x == 0 && tid == 0) {
        gb[0] = lo;
        gb[G] = end;
    }
    __syncthreads();
    if (W == 0) return;
    // groups of this block: t_m in (c_K0, c_K1], and t_m = 0 in block 0
    const u64 cK0 = cs[0], cK1 = cs[nloc];
    u64 m_lo = blockIdx.x == 0 ? 1 : muldiv_floor(cK0 + 1, G, W - 1, W);
    // last m with t_m <= c_K1: floor(((c + 1) G - 1) / W) = ceil((c + 1) G / W) - 1
    u64 m_hi = muldiv_floor(cK1 + 1, G, W - 1, W) - 1;
    if (m_lo < 1) m_lo = 1;
    if (m_hi > (u64)G - 1) m_hi = (u64)G - 1;
    for (u64 m = m_lo + tid; m <= m_hi; m += GC_T) {
        const u64 tm = muldiv_floor(W, m, 0, G);
        // first j in [0, nloc] with cs[j] >= tm; the bucket index is K0 + j
        u32 a = 0, len = nloc + 1;
        while (len > 0) {
            const u32 half = len >> 1;
            if (cs[a + half] < tm) {
                a += half + 1;
                len -= half + 1;
            } else {
                len = half;
            }
        }
        u64 v = lo + (K0 + a) * bw;
        gb[m] = v > end ? end : v;
    }
}

u64 *direct_groups(Ctx &c, Scratch &S, const u64 *A, u32 na, const u64 *B, u32 nb, u64 lo, u64 end, u32 G,
                   u32 grid_l, u64 products, u32 win, u32 cost_row, u32 cost_window, u64 nbk_max)
{
    // cost model: a grid point of the pp-matrix stands for products / ng
    // term products; a bucket also carries its share of the window costs
    // (rows staged and per-window work, k_hist_rows)
    const GridShape gs = grid_shape(na, nb, grid_l ? grid_l : 1);
    const u64 ng = gs.total;
    const u64 span = end - lo;
    const u64 nbk = span < nbk_max ? span : nbk_max;
    const u64 bw = (span + nbk - 1) / nbk;
    const u32 nparts = (u32)((nbk + HB - 1) / HB);
    u64 *hist = S.get<u64>(nbk), *part = S.get<u64>(nparts);
    PM_CUDA(cudaMemsetAsync(hist, 0, nbk * 8, c.s));
    const u64 wg = products / ng + 1;
    k_grid_hist<<<(unsigned)((ng + 255) / 256), 256, 0, c.s>>>(A, na, B, nb, gs, lo, bw, nbk, wg, hist);
    PM_LAUNCHED(c);
    u64 *kw = S.get<u64>(nbk);
    const u64 w = win ? win : 1;
    k_hist_rows<<<nparts, HB, 0, c.s>>>(A, na, B, nb, lo, bw, w, nbk, cost_row, cost_window, hist, kw, part);
    PM_LAUNCHED(c);
    u64 *gb = S.get<u64>(G + 1);
    const u32 ncut = (u32)((nbk + GC_BUCKETS - 1) / GC_BUCKETS);
    k_group_cut<<<ncut, GC_T, 0, c.s>>>(hist, part, nparts, nbk, G, lo, end, bw, gb);
    PM_LAUNCHED(c);
    // one refinement: charge narrow groups their whole window, cut again
    k_hist_narrow<<<nparts, HB, 0, c.s>>>(gb, G, lo, bw, w, nbk, kw, hist, part);
    PM_LAUNCHED(c);
    k_group_cut<<<ncut, GC_T, 0, c.s>>>(hist, part, nparts, nbk, G, lo, end, bw, gb);
    PM_LAUNCHED(c);
    return gb;
}

static int acc_policy(int kind, u64 min_n, int requested);

// the direct kernel's accumulator: three normalised limbs by default (exact
// for any operand sizes), or the one asked for
static int direct_acc_policy(int kind, u64 min_n, int requested)
{
    if (kind == PM_COEF_M61 && (requested == PM_ACC_AUTO || requested == PM_ACC_LIMBS3)) return ACC_L3;
    return acc_policy(kind, min_n, requested);
}

static int acc_policy(int kind, u64 min_n, int requested)
{
    if (kind == PM_COEF_I64_ACC192) return ACC_I192;
    if (kind != PM_COEF_M61) return ACC_I128;
    if (requested == PM_ACC_WIDE) return ACC_W64;
    if (requested == PM_ACC_LIMBS) {
        if (min_n > 65537) throw Error(PM_EINVAL, "limb accumulators need min(n_f, n_g) <= 65537");
        return ACC_L16;
    }
    return min_n <= 65537 ? ACC_L16 : ACC_W64;
}

static u32 acc_bytes(int acc) { return (acc == ACC_W64 || acc == ACC_L3) ? 12 : (acc == ACC_I192 ? 24 : 16); }

size_t direct_smem_bytes(u32 slots, int kind, u64 min_n, int requested)
{
    (void)slots;  // the accumulator arrays always take their full stride
    const u32 b = acc_bytes(direct_acc_policy(kind, min_n, requested));
    return (size_t)acc_stride(b) * b + DTABLE_BYTES;
}

u32 direct_max_slots(int kind, u64 min_n, int requested)
{
    // 227 KB of opt-in shared memory per CTA, minus tables and static use
    return acc_stride(acc_bytes(direct_acc_policy(kind, min_n, requested)));
}

template <class K>
static void set_smem(K kernel, size_t bytes)
{
    PM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}


void launch_direct(Ctx &c, Scratch &S, DirectArgs &a, u32 slots, int kind, int requested, u64 end, u32 cost_row,
                   u32 cost_window, cudaEvent_t ev_k0, cudaEvent_t ev_k1)
{
    const u32 G = a.ngroups;
    // window boundaries W (at most G + span / slots + 1 of them)
    u64 *nw = S.get<u64>(G);
    u64 *wpos = S.get<u64>(G + 1);
    k_window_count<<<(G + 255) / 256, 256, 0, c.s>>>(a.gb, G, slots, nw);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, nw, wpos, G);
    const u64 nbmax = G + (end - a.lo + slots - 1) / slots + 1;
    u64 *W = S.get<u64>(nbmax);
    k_window_bounds<<<(G + 255) / 256, 256, 0, c.s>>>(a.gb, G, slots, wpos, W);
    PM_LAUNCHED(c);
    if (nbmax * a.na > (2ull << 30)) throw Error(PM_ENOMEM, "edge table too large");
    a.W = W;
    a.wpos = wpos;
    a.E = S.get<u32>(nbmax * a.na);
    a.i0s = S.get<u32>(nbmax);
    a.i1s = S.get<u32>(nbmax);
    a.cnt = S.get<u64>(nbmax);

    // FindEdge at every boundary
    const unsigned fgrid = (unsigned)(nbmax < (u64)c.sm_count * 4 ? nbmax : (u64)c.sm_count * 4);
    // g's keys in shared memory when they fit in 200 KB, the row edges too
    // when both fit (two CTAs of 1024 threads share an SM up to ~113 KB each)
    auto fe_smem = [&](size_t kbytes, u32 &stage, u32 &stage_e) {
        const size_t sb = (size_t)a.nb * kbytes, se = (size_t)a.na * 4;
        stage = sb <= 200 * 1024;
        const size_t sbs = stage ? (sb + 15) / 16 * 16 : 0;
        stage_e = sbs + se <= 200 * 1024;
        return sbs + (stage_e ? se : 0);
    };
    u32 stage = 0, stage_e = 0;
    if (a.A32) {
        const size_t bytes = fe_smem(4, stage, stage_e);
        set_smem(k_find_edge<u32>, bytes);
        k_find_edge<u32><<<fgrid, DT, bytes, c.s>>>(a.A32, a.B32, a.na, a.nb, W, wpos + G, a.E, a.i0s, a.i1s,
                                                    a.cnt, stage, stage_e);
    } else {
        const size_t bytes = fe_smem(8, stage, stage_e);
        set_smem(k_find_edge<u64>, bytes);
        k_find_edge<u64><<<fgrid, DT, bytes, c.s>>>(a.A, a.B, a.na, a.nb, W, wpos + G, a.E, a.i0s, a.i1s, a.cnt,
                                                    stage, stage_e);
    }
    PM_LAUNCHED(c);

    // windows in descending cost, per-window result counts, the counter
    a.order = S.get<u32>(nbmax);
    a.ucount = S.get<u64>(nbmax + 1);
    a.wnext = S.get<u32>(1);
    a.nwin_max = nbmax;
    PM_CUDA(cudaMemsetAsync(a.ucount, 0, (nbmax + 1) * 8, c.s));
    PM_CUDA(cudaMemsetAsync(a.wnext, 0, 4, c.s));
    k_window_order<<<1, 1024, 0, c.s>>>(a.cnt, a.i0s, a.i1s, wpos + G, cost_row, cost_window, a.order);
    PM_LAUNCHED(c);

    // accumulate: persistent CTAs, one per SM; mod-p kinds read g's
    // coefficients split for m61_mul_split
    const int acc = direct_acc_policy(kind, a.na < a.nb ? a.na : a.nb, requested);
    if (acc == ACC_L3) {
        uint4 *rec = S.get<uint4>(a.nb);
        k_col_rec<<<(a.nb + 255) / 256, 256, 0, c.s>>>(a.Bc, a.B32, rec, a.nb);
        PM_LAUNCHED(c);
        a.Brec = rec;
    } else if (acc == ACC_W64 || acc == ACC_L16) {
        u64 *bs = S.get<u64>(a.nb);
        k_split_col<<<(a.nb + 255) / 256, 256, 0, c.s>>>(a.Bc, bs, a.nb);
        PM_LAUNCHED(c);
        a.Bc = bs;
    }
    const size_t bytes = (size_t)acc_stride(acc_bytes(acc)) * acc_bytes(acc) + DTABLE_BYTES;
    const unsigned grid = (unsigned)(nbmax < (u64)c.sm_count ? nbmax : (u64)c.sm_count);
    if (ev_k0) PM_CUDA(cudaEventRecord(ev_k0, c.s));
    if (acc == ACC_W64) {
        set_smem(k_direct<ACC_W64>, bytes);
        k_direct<ACC_W64><<<grid, DT, bytes, c.s>>>(a, slots);
    } else if (acc == ACC_L16) {
        set_smem(k_direct<ACC_L16>, bytes);
        k_direct<ACC_L16><<<grid, DT, bytes, c.s>>>(a, slots);
    } else if (acc == ACC_L3) {
        set_smem(k_direct<ACC_L3>, bytes);
        k_direct<ACC_L3><<<grid, DT, bytes, c.s>>>(a, slots);
    } else if (acc == ACC_I128) {
        set_smem(k_direct<ACC_I128>, bytes);
        k_direct<ACC_I128><<<grid, DT, bytes, c.s>>>(a, slots);
    } else {
        set_smem(k_direct<ACC_I192>, bytes);
        k_direct<ACC_I192><<<grid, DT, bytes, c.s>>>(a, slots);
    }
    PM_LAUNCHED(c);
    if (ev_k1) PM_CUDA(cudaEventRecord(ev_k1, c.s));
}

// ---------------------------------------------------------------------------
// Hashed windows: products whose result is sparse in a large rank box.
//
// A direct-addressed window holds one slot per rank, so a sparse box needs
// so many windows that the FindEdge table (a row per window) and the row
// staging per window explode.  Here a window may span up to 2^31 ranks; its
// distinct result monomials go to a shared-memory hash table (HT slots,
// linear probing, bounded), and FindEdge is done inside the kernel: for the
// window's two boundaries every row's column edges move up from where the
// CTA's previous window left them (a CTA takes runs of consecutive windows
// and the windows ascend, so the edges only rise, Sec. 2) by a short gallop
// per row, the rows independent of one another; rows new to the CTA start
// from column 0.  Each thread then inserts the products of its rows (tid,
// tid + 1024, ...) directly.  Emission sorts the
// occupied slots by rank (block_sort_interval) and writes the window's
// terms in order.  A window with more than HT_LOAD distinct monomials (or a
// probe run longer than HT_PROBES) is abandoned and reported; the host
// splits it in four and runs the parts in the next round.
// ---------------------------------------------------------------------------

constexpr u32 HT = 4096, HT_BITS = 12;
constexpr u32 HWIN_RUN = 16;  // consecutive windows a CTA takes at a time
// a window may fill 3968 of the 4096 slots (probe runs up to 256): fewer,
// fuller windows beat shorter probe runs here
constexpr u32 HT_LOAD = 3968;
constexpr u32 HT_PROBES = 256;
constexpr u32 HEMPTY = 0xFFFFFFFFu;
constexpr u64 HFAILED = ~0ull;

struct HashArgs {
    const u64 *A, *Ac, *B, *Bc;  // canonical f and g: ranks (sorted) and coefficients
    const u32 *B32;              // low 32 bits of g's ranks
    u32 na, nb;
    const u64 *wlo, *whi;        // the round's windows (rank bounds)
    u32 nwin;
    u32 *E2;                     // per CTA: each row's upper column edge in its last window (na words, by row)
    u32 *RL;                     // per CTA: the window's rows with products and their lower edges, in any order (2 na words)
    u64 *okey, *ocoef;           // window w's terms at w * HT (coefficient words: words)
    u64 *ucount;                 // terms of window w, or HFAILED
    u32 *wnext;                  // window counter
    Layout L;
    u32 words;
    u32 mixed;                   // wide accumulator chosen by the library: windows may use the limbs
    const u32 *abort;
};

template <int ACC>
__global__ void __launch_bounds__(DT, 1) k_hash(HashArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 s_next, s_count, s_over, s_rows[2], s_nlist, s_take;
    using HA = Acc<ACC, HT>;
    // when the library chose the wide accumulator (operands above 65537
    // terms), a window switches to the four-limb one if at most 65537 rows
    // have products in it: a slot takes at most one product per row, so the
    // limb counters cannot overflow, and their fire-and-forget reductions
    // are cheaper than the wide one's returned add.  Both lay out on the
    // same 16 bytes per slot.
    constexpr bool HYB = ACC == ACC_W64;
    using HL = Acc<ACC_L16, HT>;
    constexpr u32 SLOT_B = HYB ? HL::bytes : HA::bytes;
    u32 *keys = (u32 *)smem;
    HA acc;
    HL acc16;
    acc.carve(smem + HT * 4);
    acc16.carve(smem + HT * 4);
    unsigned char *sb_ = smem + HT * 4 + (size_t)HT * SLOT_B;
    u64 *kA = (u64 *)sb_, *kB = kA + HT;
    uint16_t *iA = (uint16_t *)(kB + HT), *iB = iA + HT;
    u32 *hist = (u32 *)(iB + HT);  // HT_HIST words
    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (a.abort && *a.abort) return;
    u32 *E2 = a.E2 + (size_t)blockIdx.x * a.na;
    u32 *RL = a.RL + (size_t)blockIdx.x * 2 * a.na;
    const u64 bmin = a.B[0], bmax = a.B[a.nb - 1];
    // clear a slot: in the mixed case every byte of its 16 (both layouts)
    auto zero_slot = [&](u32 x) {
        if (HYB) acc16.zero(x);
        else acc.zero(x);
    };
    for (u32 x = tid; x < HT; x += DT) {
        keys[x] = HEMPTY;
        zero_slot(x);
    }
    if (tid == 0) {
        s_rows[0] = 0;
        s_rows[1] = 0;
    }
    u32 pi1 = 0;   // rows below pi1 hold edges of an earlier window of this CTA
    for (;;) {
        if (tid == 0) s_next = atomicAdd(a.wnext, HWIN_RUN);
        __syncthreads();
        const u32 wbase = s_next;
        if (wbase >= a.nwin) break;
        const u32 wstop = min(wbase + HWIN_RUN, a.nwin);
        for (u32 wk = wbase; wk < wstop; wk++) {
        const u64 lo = a.wlo[wk], hi = a.whi[wk];
        const u32 span = (u32)(hi - lo);
        if (tid == 0) {
            s_count = 0;
            s_over = 0;
            s_nlist = 0;
            s_take = 0;
            // rows reaching the window, from the last window's rows
            s_rows[0] = lo > bmax ? gallop_up_k(a.A, a.na, s_rows[0], lo - bmax) : s_rows[0];
            s_rows[1] = hi > bmin ? gallop_up_k(a.A, a.na, s_rows[1], hi - bmin) : s_rows[1];
        }
        __syncthreads();
        const u32 i0 = s_rows[0], i1 = s_rows[1];
        // FindEdge for both boundaries: each row's edges rise from its edge
        // at the last window's top (0 for rows new to this CTA); the thread
        // lists its rows that have products in the window
        // (the warp's rows with products are appended to the list with one
        // atomic per warp and step)
        for (u32 r0 = i0 + (tid & ~31u); r0 < i1; r0 += DT) {
            const u32 r = r0 + lane;
            bool has = false;
            u32 jl = 0;
            if (r < i1) {
                const u64 ar = a.A[r];
                const bool known = r < pi1;
                const u32 js = known ? E2[r] : 0u;
                jl = gallop_up_k(a.B, a.nb, js, lo > ar ? lo - ar : 0);
                const u32 jh = gallop_up_k(a.B, a.nb, js, hi > ar ? hi - ar : 0);
                // most rows have no product in the window and keep their
                // edge: no store for them
                if (jh != js || !known) E2[r] = jh;
                has = jh > jl;
            }
            const u32 bal = __ballot_sync(0xffffffffu, has);
            u32 at = 0;
            if (lane == 0 && bal) at = atomicAdd(&s_nlist, (u32)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (has) {
                const u32 x = at + __popc(bal & ((1u << lane) - 1u));
                RL[2 * x] = r;
                RL[2 * x + 1] = jl;
            }
        }
        if (i1 > pi1) pi1 = i1;
        __syncthreads();
        // the products: warps take the listed rows from a counter, and the
        // 32 lanes of a warp insert a row's products together (consecutive
        // columns: coalesced loads, and no two lanes of one step share a
        // monomial).  A window's rows hold tens of products each and very
        // unevenly, so a thread per row would leave the block waiting for
        // its busiest thread.
        const volatile u32 *over = &s_over;
        const u32 nlist = s_nlist;
        const bool limbs = HYB && a.mixed && nlist <= 65537;
        constexpr u32 TAKE = 4;  // rows per claim
        for (;;) {
            u32 t0 = 0;
            if (lane == 0) t0 = *over ? nlist : atomicAdd(&s_take, TAKE);
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            if (t0 >= nlist) break;
            for (u32 t = t0; t < min(t0 + TAKE, nlist); t++) {
            const u32 i = RL[2 * t], jl = RL[2 * t + 1], jh = E2[i];
            const u32 ra = (u32)a.A[i] - (u32)lo;
            const u64 ca = a.Ac[i];
            for (u32 j = jl + lane; j < jh; j += 32) {
                const u32 key = ra + __ldg(a.B32 + j);  // rank - lo, below span
                const u64 gc = __ldg(a.Bc + j);
                // linear probing from a multiplicative hash of the rank
                u32 h = (key * 2654435761u) >> (32 - HT_BITS);
                bool done = false;
                for (u32 probe = 0; probe < HT_PROBES; probe++) {
                    const u32 k = keys[h];
                    if (k == key) {
                        done = true;
                        break;
                    }
                    if (k == HEMPTY) {
                        const u32 old = atomicCAS(&keys[h], HEMPTY, key);
                        if (old == HEMPTY) {
                            if (atomicAdd(&s_count, 1u) >= HT_LOAD) s_over = 1;
                        }
                        if (old == HEMPTY || old == key) {
                            done = true;
                            break;
                        }
                    }
                    h = (h + 1) & (HT - 1);
                }
                if (!done) {
                    s_over = 1;
                    break;
                }
                if (limbs) acc16.add(h, ca, gc);
                else acc.add(h, ca, gc);
            }
            }
        }
        __syncthreads();
        if (s_over) {
            // abandoned: report it, clear the table for the next window
            for (u32 x = tid; x < HT; x += DT) {
                keys[x] = HEMPTY;
                zero_slot(x);
            }
            if (tid == 0) a.ucount[wk] = HFAILED;
            __syncthreads();
            continue;
        }
        // emission: the occupied slots with non-zero values, sorted by rank
        constexpr u32 PER = HT / DT;
        u32 mine = 0;
        u32 nzf = 0;
#pragma unroll
        for (u32 q = 0; q < PER; q++) {
            const u32 x = tid * PER + q;
            u64 v0, v1, v2;
            if (keys[x] != HEMPTY && (limbs ? acc16.finalize(x, v0, v1, v2) : acc.finalize(x, v0, v1, v2))) {
                nzf |= 1u << q;
                mine++;
            }
        }
        u64 nall;
        u64 pos = block_exclusive_scan(mine, nall, ws);
#pragma unroll
        for (u32 q = 0; q < PER; q++) {
            const u32 x = tid * PER + q;
            if ((nzf >> q) & 1u) {
                kA[pos] = keys[x];
                iA[pos] = (uint16_t)x;
                pos++;
            }
        }
        __syncthreads();
        const u32 n = (u32)nall;
        block_sort_interval<DT, HT / DT>(kA, iA, kB, iB, n, 0, span ? span - 1 : 0, hist, ws);
        const u64 obase = (u64)wk * HT;
        for (u32 q = tid; q < n; q += DT) {
            const u32 x = iA[q];
            u64 v0, v1, v2;
            if (limbs) acc16.take(x, v0, v1, v2);
            else acc.take(x, v0, v1, v2);
            a.okey[obase + q] = rank_to_key(a.L, lo + kA[q]);
            constexpr u32 W = HA::words;
            a.ocoef[W * (obase + q)] = v0;
            if (W > 1) a.ocoef[W * (obase + q) + 1] = v1;
            if (W > 2) a.ocoef[W * (obase + q) + 2] = v2;
        }
        __syncthreads();
        for (u32 x = tid; x < HT; x += DT) {
            keys[x] = HEMPTY;
            zero_slot(x);
        }
        if (tid == 0) a.ucount[wk] = n;
        __syncthreads();
        }
    }
}

// each finished window's terms to their place in the result (the windows'
// scratch buffers differ by round, so a slice carries its source pointers)
__global__ void k_hash_gather(const u64 *__restrict__ kptr, const u64 *__restrict__ cptr, const u64 *__restrict__ dst,
                              const u64 *__restrict__ cnt, u32 nslices, u32 words, u64 *__restrict__ hkey,
                              u64 *__restrict__ hcoef)
{
    for (u32 k = blockIdx.x; k < nslices; k += gridDim.x) {
        const u64 *sk = (const u64 *)kptr[k], *sc = (const u64 *)cptr[k];
        const u64 d0 = dst[k], n = cnt[k];
        for (u64 t = threadIdx.x; t < n; t += blockDim.x) {
            hkey[d0 + t] = sk[t];
            for (u32 q = 0; q < words; q++) hcoef[words * (d0 + t) + q] = sc[words * t + q];
        }
    }
}

// sort histogram: the bucket sort's 4096 words or, for its radix fallback,
// 256 per warp
constexpr u32 HT_HIST = BUCKETS > DW * 256 ? BUCKETS : DW * 256;

constexpr size_t HASH_SMEM(u32 acc_bytes_)
{
    return (size_t)HT * 4 + (size_t)HT * acc_bytes_ + (size_t)HT * (8 + 8 + 2 + 2) + HT_HIST * 4;
}

u64 hash_product(Ctx &c, Scratch &S, const HashInputs &in, int kind, int requested, u64 lo, u64 end, u64 products,
                 u64 *hkey, u64 *hcoef, u64 cap, u32 *rounds_out, u64 *windows_out)
{
    const u32 words = kind == PM_COEF_M61 ? 1 : (kind == PM_COEF_I64_ACC192 ? 3 : 2);
    const int acc = acc_policy(kind, in.na < in.nb ? in.na : in.nb, requested);
    // first windows: cost-balanced by term products (no window terms),
    // about products / (4 HT) of them (at most 2^20), at least 4 per SM;
    // then no window wider than 2^31 ranks.  Small first windows overflow
    // less often, and an overflowing window's inserted products are lost
    u64 G0 = products / ((u64)HT * 4);
    if (G0 < (u64)c.sm_count * 4) G0 = (u64)c.sm_count * 4;
    if (G0 > end - lo) G0 = end - lo;
    if (G0 > (1u << 20)) G0 = 1u << 20;
    u32 l = 1;
    while ((u64)(l + 1) * (l + 1) < 256ull * G0 && l < 4096) l++;
    const u64 *gb = direct_groups(c, S, in.A, in.na, in.B, in.nb, lo, end, (u32)G0, l, products, 1u, 0u, 0u,
                                  1ull << 20);
    std::vector<u64> hgb(G0 + 1);
    PM_CUDA(cudaMemcpyAsync(hgb.data(), gb, (G0 + 1) * 8, cudaMemcpyDeviceToHost, c.s));
    c.sync();
    std::vector<u64> wl, wh;
    for (u64 g = 0; g < G0; g++) {
        for (u64 x = hgb[g]; x < hgb[g + 1];) {
            const u64 y = std::min(hgb[g + 1], x + (1ull << 31));
            wl.push_back(x);
            wh.push_back(y);
            x = y;
        }
    }
    struct Done {
        u64 lo, n;
        const u64 *k, *cf;
    };
    std::vector<Done> done;
    u32 *E2 = S.get<u32>((size_t)c.sm_count * in.na);
    u32 *RL = S.get<u32>((size_t)c.sm_count * 2 * in.na);
    // the wide accumulator's windows may use the four-limb layout (16 bytes)
    const size_t smem = HASH_SMEM(acc == ACC_W64 ? 16u : acc_bytes(acc));
    u32 rounds = 0;
    while (!wl.empty()) {
        if (++rounds > 40) throw Error(PM_ECUDA, "hash windows did not converge");
        const u32 nw = (u32)wl.size();
        if (windows_out) *windows_out += nw;
        u64 *dlo = S.get<u64>(nw), *dhi = S.get<u64>(nw), *cnt = S.get<u64>(nw);
        u64 *skey = S.get<u64>((size_t)nw * HT), *scoef = S.get<u64>((size_t)nw * HT * words);
        u32 *wnext = S.get<u32>(1);
        PM_CUDA(cudaMemcpyAsync(dlo, wl.data(), nw * 8ull, cudaMemcpyHostToDevice, c.s));
        PM_CUDA(cudaMemcpyAsync(dhi, wh.data(), nw * 8ull, cudaMemcpyHostToDevice, c.s));
        PM_CUDA(cudaMemsetAsync(wnext, 0, 4, c.s));
        HashArgs h;
        memset(&h, 0, sizeof(h));
        h.A = in.A;
        h.Ac = in.Ac;
        h.B = in.B;
        h.Bc = in.Bc;
        h.B32 = in.B32;
        h.na = in.na;
        h.nb = in.nb;
        h.wlo = dlo;
        h.whi = dhi;
        h.nwin = nw;
        h.E2 = E2;
        h.RL = RL;
        h.okey = skey;
        h.ocoef = scoef;
        h.ucount = cnt;
        h.wnext = wnext;
        h.L = in.L;
        h.words = words;
        h.mixed = acc == ACC_W64 && requested != PM_ACC_WIDE ? 1u : 0u;
        const unsigned grid = (unsigned)std::min<u64>(nw, (u64)c.sm_count);
        if (acc == ACC_W64) {
            set_smem(k_hash<ACC_W64>, smem);
            k_hash<ACC_W64><<<grid, DT, smem, c.s>>>(h);
        } else if (acc == ACC_L16) {
            set_smem(k_hash<ACC_L16>, smem);
            k_hash<ACC_L16><<<grid, DT, smem, c.s>>>(h);
        } else if (acc == ACC_I128) {
            set_smem(k_hash<ACC_I128>, smem);
            k_hash<ACC_I128><<<grid, DT, smem, c.s>>>(h);
        } else {
            set_smem(k_hash<ACC_I192>, smem);
            k_hash<ACC_I192><<<grid, DT, smem, c.s>>>(h);
        }
        PM_LAUNCHED(c);
        std::vector<u64> hc(nw);
        PM_CUDA(cudaMemcpyAsync(hc.data(), cnt, nw * 8ull, cudaMemcpyDeviceToHost, c.s));
        c.sync();
        std::vector<u64> nl, nh;
        for (u32 k = 0; k < nw; k++) {
            if (hc[k] == HFAILED) {
                // four parts of equal rank width (fewer when narrower)
                const u64 span = wh[k] - wl[k];
                if (span < 2) throw Error(PM_ECUDA, "hash window of one monomial overflowed");
                const u64 parts = span < 4 ? span : 4;
                for (u64 q = 0; q < parts; q++) {
                    nl.push_back(wl[k] + span * q / parts);
                    nh.push_back(wl[k] + span * (q + 1) / parts);
                }
            } else if (hc[k]) {
                done.push_back(Done{wl[k], hc[k], skey + (size_t)k * HT, scoef + (size_t)k * HT * words});
            }
        }
        wl.swap(nl);
        wh.swap(nh);
    }
    if (rounds_out) *rounds_out = rounds;
    // the windows in rank order, concatenated
    std::sort(done.begin(), done.end(), [](const Done &x, const Done &y) { return x.lo < y.lo; });
    u64 n_out = 0;
    for (const Done &d : done) n_out += d.n;
    const u32 ns = (u32)done.size();
    // the gather's tables are taken before the capacity check, so a call
    // without room for the result (the workspace size query) takes the
    // same scratch as one with room
    u64 *dsrc = S.get<u64>(ns), *dsrcc = S.get<u64>(ns), *ddst = S.get<u64>(ns), *dcn = S.get<u64>(ns);
    if (n_out > cap || !hkey) return n_out;
    std::vector<u64> src(ns), srcc(ns), dst(ns), cn(ns);
    u64 run = 0;
    for (u32 k = 0; k < ns; k++) {
        src[k] = (u64)(uintptr_t)done[k].k;
        srcc[k] = (u64)(uintptr_t)done[k].cf;
        dst[k] = run;
        cn[k] = done[k].n;
        run += done[k].n;
    }
    PM_CUDA(cudaMemcpyAsync(dsrc, src.data(), ns * 8ull, cudaMemcpyHostToDevice, c.s));
    PM_CUDA(cudaMemcpyAsync(dsrcc, srcc.data(), ns * 8ull, cudaMemcpyHostToDevice, c.s));
    PM_CUDA(cudaMemcpyAsync(ddst, dst.data(), ns * 8ull, cudaMemcpyHostToDevice, c.s));
    PM_CUDA(cudaMemcpyAsync(dcn, cn.data(), ns * 8ull, cudaMemcpyHostToDevice, c.s));
    if (ns) {
        k_hash_gather<<<std::min<u32>(ns, 65535u), 256, 0, c.s>>>(dsrc, dsrcc, ddst, dcn, ns, words, hkey, hcoef);
        PM_LAUNCHED(c);
    }
    c.sync();  // the host vectors above must outlive the copies
    return n_out;
}

}  // namespace pm
