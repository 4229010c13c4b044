// K-f: many independent products in one device pass (include/polymul.h,
// pm_batch_*), captured once in a CUDA graph.
//
// Alg. 1 of the paper applied to every product of the batch at once, with
// no host synchronisation between the steps:
//   B1  one CTA per operand: pack (Sec. 7), sort, combine repeated
//       monomials, drop zeros (the sorted distributed format of Sec. 2);
//   B2  one CTA per product: the error rules, then the first step of
//       Alg. 1 -- the almost regular grid of Sec. 5 over the product's
//       pp-matrix, sorted -- gives splitters S; consecutive splitters bound
//       left-closed, right-open ranges with about `target` term products;
//   B3  a persistent kernel: each CTA takes work items (a run of
//       consecutive ranges of one product) from a device counter -- the
//       dynamic scheduling of Sec. 2 -- keeps per-row column cursors in
//       shared memory so FindEdge for the next range is a short gallop, and
//       sorts and reduces each range in shared memory (ranges with more
//       products than fit are bisected by key);
//   B4  one CTA per product sizes its result, checks the capacity and
//       places its ranges in ascending order; then warps on all SMs copy
//       the ranges into the callers' outputs.
// No two CTAs write the same output term.  A product whose output capacity
// holds all its term products writes each range's terms straight into h, at
// the number of term products below the range (the sum of the rows' column
// cursors at the range's start): when no two products share a monomial --
// the usual case of sparse supports -- that is the term's final place, and
// B4 only checks it; otherwise B4 lists the product's output in units of
// CMP_CH terms and CTAs on all SMs move them left into place (kb_compact).  Other
// products claim scratch for their range results from a device bump
// counter (bounded by their term products) and B4 copies them.
#include <cstring>
#include <mutex>
#include <vector>

#include "pm_blocksort.cuh"
#include "pm_partition.cuh"

namespace pm {

constexpr u32 BT_MAX_TERMS = PM_BATCH_MAX_TERMS;  // per operand
constexpr int CAN_T = 1024;                       // B1 threads
constexpr int CAN_IPT = 8;                        // 8192 items
constexpr int PLAN_T = 1024;                      // B2 threads
constexpr u32 PLAN_SAMPLES = 8192;
// Products sorted per piece.  A product takes 8 + 8 (keys) + 2 + 2
// (indexes) + 8 per coefficient word bytes of shared memory, so a batch
// whose products are all mod p (one word) fits 4096, the others 3072.
__host__ __device__ constexpr u32 rng_chunk(u32 cw) { return cw == 1 ? 4096u : 3072u; }
// term products per range unless tuned (measured on the 4096-product sparse
// batch: one-word 126 -> 116 ms at 2048 with the wider chunk, 110.5 ms at
// 3072, no better above)
__host__ __device__ constexpr u32 rng_target_default(u32 cw) { return cw == 1 ? 3072u : 2048u; }
constexpr int FIN_T = 512;

// per-product descriptor (device); fields after `out_` are written by the
// kernels
struct BDesc {
    Layout L;
    i64 kind;
    const u32 *fe;
    const u64 *fc;
    const u32 *ge;
    const u64 *gc;
    u64 *hkey;
    u64 *hcoef;
    u64 hcap;
    u32 nf, ng;
    u64 op_off;   // canonical f at op_off, g at op_off + nf
    u64 rg_off;   // ranges [rg_off, rg_off + rcap)
    u32 rcap;
    u32 direct;   // results go straight to h (h.cap >= n_f n_g): see kb_ranges
    // out_
    u32 status;   // ST_* bits
    u32 cf, cg, nranges;
    u64 n_out;
    u64 cmp_base;  // first compaction unit (kb_compact) of a direct product that moves
    u32 maxe[2][PM_MAX_VARS];
    u64 maxabs[2];
};

struct BArgs {
    BDesc *D;
    u32 count;
    u64 *ck, *cc;                 // canonical operand keys / coefficients
    u64 *rlo, *rhi, *rbase, *rcount;
    const u32 *item_prod, *item_first;
    u32 nitems;
    u32 *work;                    // work counter
    u64 *bump;                    // output scratch counter
    u64 *skey, *scoef;            // output scratch; coefficient words per term: cw
    u32 cw;
    u32 maxt;                     // largest operand of the batch, rounded up to 4096 or 8192 terms
    u32 target;                   // term products per range
    u32 per_item;                 // ranges per work item
    u64 rg_total;                 // range slots of the batch
    u32 *uprod, *uflag;           // compaction units: product, "sources read" flag
    u32 *ucount;                  // [0] units listed by kb_finish, [1] units taken by kb_compact
};

// ---------------------------------------------------------------------------
// B1: canonical operands
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(CAN_T) kb_canon(BArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u64 orv, andv;
    __shared__ u32 maxe[PM_MAX_VARS];
    __shared__ u64 maxabs;
    const u32 p = blockIdx.x >> 1, side = blockIdx.x & 1, tid = threadIdx.x;
    BDesc &d = a.D[p];
    const u32 n = side ? d.ng : d.nf;
    const u32 *exps = side ? d.ge : d.fe;
    const u64 *coefs = side ? d.gc : d.fc;
    const Layout &L = d.L;
    const int kind = (int)d.kind;
    u64 *kA = (u64 *)smem, *kB = kA + BT_MAX_TERMS;
    uint16_t *iA = (uint16_t *)(kB + BT_MAX_TERMS), *iB = iA + BT_MAX_TERMS;
    u32 *hist = (u32 *)(iB + BT_MAX_TERMS);
    if (tid == 0) {
        orv = 0;
        andv = ~0ull;
        maxabs = 0;
    }
    if (tid < PM_MAX_VARS) maxe[tid] = 0;
    __syncthreads();
    u64 o = 0, an = ~0ull;
    u32 bad = 0;
    for (u32 t = tid; t < n; t += CAN_T) {
        u64 key = 0;
        for (u32 v = 0; v < L.nv; v++) {
            const u64 e = exps[(size_t)t * L.nv + v];
            if (e >= (1ull << (L.width[v] - 1))) bad = 1;
            key |= e << L.off[v];
        }
        kA[t] = key;
        iA[t] = (uint16_t)t;
        o |= key;
        an &= key;
    }
    if (bad) atomicOr(&d.status, ST_EXP_OVERFLOW);
    atomicOr(&orv, o);
    atomicAnd(&andv, an);
    __syncthreads();
    int nbits = 0;
    for (u64 x = orv ^ andv; x; x >>= 1) nbits++;
    block_sort_pairs<CAN_T, CAN_IPT>(kA, iA, kB, iB, n, nbits, hist, ws);

    // combine runs of equal keys, drop zero sums, write in order
    u64 *ck = a.ck + d.op_off + (side ? d.nf : 0), *cc = a.cc + d.op_off + (side ? d.nf : 0);
    u32 run = 0;
    u64 ma = 0;
    for (u32 t0 = 0; t0 < n; t0 += CAN_T) {
        const u32 i = t0 + tid;
        u64 v = 0;
        bool nz = false;
        if (i < n && (i == 0 || kA[i] != kA[i - 1])) {
            if (kind == PM_COEF_M61) {
                for (u32 j = i; j < n && kA[j] == kA[i]; j++) v = m61_add(v, m61_reduce(coefs[iA[j]]));
                nz = v != 0;
            } else {
                u64 lo = 0, hi = 0;
                for (u32 j = i; j < n && kA[j] == kA[i]; j++) {
                    const u64 c = coefs[iA[j]];
                    add128(lo, hi, c, (u64)((i64)c >> 63));
                }
                if (hi != (u64)((i64)lo >> 63)) atomicOr(&d.status, ST_COEF_BOUND);
                v = lo;
                nz = (lo | hi) != 0;
                if (nz) {
                    const u64 m = (i64)lo < 0 ? (u64)0 - lo : lo;
                    ma = m > ma ? m : ma;
                }
            }
        }
        u64 cnt;
        const u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, ws);
        if (nz) {
            ck[run + pos] = kA[i];
            cc[run + pos] = v;
            for (u32 vv = 0; vv < L.nv; vv++) atomicMax(&maxe[vv], key_field(L, kA[i], vv));
        }
        run += (u32)cnt;
    }
    if (kind != PM_COEF_M61) atomicMax(&maxabs, ma);
    __syncthreads();
    if (tid == 0) {
        if (side) d.cg = run;
        else d.cf = run;
        d.maxabs[side] = maxabs;
    }
    if (tid < PM_MAX_VARS) d.maxe[side][tid] = maxe[tid];
}

// ---------------------------------------------------------------------------
// B2: error rules and ranges
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(PLAN_T) kb_plan(BArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 flag, nuniq;
    const u32 p = blockIdx.x, tid = threadIdx.x;
    BDesc &d = a.D[p];
    const Layout &L = d.L;
    if (tid == 0) {
        u32 st = d.status;
        if (!st && d.cf && d.cg) {
            for (u32 v = 0; v < L.nv; v++)
                if ((u64)d.maxe[0][v] + d.maxe[1][v] >= (1ull << (L.width[v] - 1))) st |= ST_EXP_OVERFLOW;
            if (d.kind != PM_COEF_M61) {
                const unsigned __int128 m = (unsigned __int128)d.maxabs[0] * d.maxabs[1];
                const unsigned __int128 lim = ((((unsigned __int128)1) << 127) - 1) / (d.cf < d.cg ? d.cf : d.cg);
                if (m > lim) st |= ST_COEF_BOUND;
            }
        }
        d.status = st;
        flag = (st || !d.cf || !d.cg) ? 1u : 0u;
        if (flag) d.nranges = 0;
    }
    __syncthreads();
    if (flag) return;
    const u32 cf = d.cf, cg = d.cg;
    const u64 *A = a.ck + d.op_off, *B = A + d.nf;
    const u64 lo = A[0] + B[0], end = A[cf - 1] + B[cg - 1] + 1;  // gamma_end
    const u64 P = (u64)cf * cg;
    u64 R = (P + a.target - 1) / a.target;
    if (R > d.rcap) R = d.rcap;
    if (R > PLAN_SAMPLES) R = PLAN_SAMPLES;
    u64 *rlo = a.rlo + d.rg_off, *rhi = a.rhi + d.rg_off;
    if (R <= 1) {
        if (tid == 0) {
            rlo[0] = lo;
            rhi[0] = end;
            d.nranges = 1;
        }
        return;
    }
    // Sec. 5 grid: steps floor(n/l) clamped to >= 1, alternate rows shifted
    // by floor(n_b / 2l), plus the last row and column, (l+1)^2 points.
    // About four points per range where the sample buffer allows (the
    // splitters are every fourth order statistic then, and fewer ranges
    // exceed the shared-memory chunk than with one point per range);
    // floor-divided steps can give more, so shrink l until the whole grid
    // fits the sample buffer
    const u64 Rs = 4 * R < PLAN_SAMPLES ? 4 * R : PLAN_SAMPLES;
    u32 l = 1;
    while ((u64)(l + 2) * (l + 2) <= Rs) l++;
    GridShape gsh;
    for (;;) {
        gsh = grid_shape(cf, cg, l);
        if (gsh.total <= PLAN_SAMPLES || l == 1) break;
        l--;
    }
    const u32 ns = (u32)(gsh.total < PLAN_SAMPLES ? gsh.total : PLAN_SAMPLES);
    u64 *kA = (u64 *)smem, *kB = kA + PLAN_SAMPLES;
    uint16_t *iA = (uint16_t *)(kB + PLAN_SAMPLES), *iB = iA + PLAN_SAMPLES;
    u32 *hist = (u32 *)(iB + PLAN_SAMPLES);
    for (u32 q = tid; q < ns; q += PLAN_T) {
        u64 i, j;
        grid_point(gsh, cf, cg, q, i, j);
        kA[q] = A[i] + B[j];
        iA[q] = (uint16_t)q;
    }
    __syncthreads();
    block_sort_pairs<PLAN_T, PLAN_SAMPLES / PLAN_T>(kA, iA, kB, iB, ns, varying_bits(lo, end - 1), hist, ws);
    // distinct samples strictly inside (lo, end): kB[0..nuniq)
    u32 run = 0;
    for (u32 t0 = 0; t0 < ns; t0 += PLAN_T) {
        const u32 q = t0 + tid;
        const bool keep = q < ns && kA[q] > lo && kA[q] < end && (q == 0 || kA[q] != kA[q - 1]);
        u64 cnt;
        const u64 pos = block_exclusive_scan(keep ? 1 : 0, cnt, ws);
        if (keep) kB[run + pos] = kA[q];
        run += (u32)cnt;
    }
    if (tid == 0) nuniq = run;
    __syncthreads();
    // R - 1 splitters at evenly spaced order statistics, deduplicated
    const u32 m = nuniq;
    const u32 want = (u32)R - 1 < m ? (u32)R - 1 : m;
    run = 0;
    for (u32 t0 = 0; t0 < want; t0 += PLAN_T) {
        const u32 k = t0 + tid;
        u64 s = 0;
        bool keep = false;
        if (k < want) {
            const u32 at = (u32)(((u64)(k + 1) * m) / (want + 1));
            s = kB[at < m ? at : m - 1];
            const u32 atp = k ? (u32)(((u64)k * m) / (want + 1)) : 0;
            keep = k == 0 || s != kB[atp < m ? atp : m - 1];
        }
        u64 cnt;
        const u64 pos = block_exclusive_scan(keep ? 1 : 0, cnt, ws);
        if (keep) rlo[1 + run + pos] = s;  // splitter k starts range k + 1
        run += (u32)cnt;
    }
    __syncthreads();
    const u32 nr = run + 1;
    for (u32 k = tid; k < nr; k += PLAN_T) {
        if (k == 0) rlo[0] = lo;
        rhi[k] = k + 1 < nr ? rlo[k + 1] : end;
    }
    if (tid == 0) d.nranges = nr;
}

// ---------------------------------------------------------------------------
// B3: ranges, persistent
// ---------------------------------------------------------------------------

// smallest j' >= j with B[j'] >= x (n if none), B sorted
__device__ __forceinline__ u32 gallop_up(const u64 *B, u32 n, u32 j, u64 x)
{
    if (j >= n || B[j] >= x) return j;
    u32 lo = j;  // B[lo] < x
    u32 step = 1;
    for (;;) {
        const u32 probe = lo + step;
        if (probe >= n || B[probe] >= x) {
            // answer in (lo, min(probe, n)]
            const u32 top = probe < n ? probe : n;
            u32 a = lo + 1, len = top - a;
            while (len > 0) {
                const u32 half = len >> 1;
                if (B[a + half] < x) {
                    a += half + 1;
                    len -= half + 1;
                } else {
                    len = half;
                }
            }
            return a;
        }
        lo = probe;
        step <<= 1;
    }
}

struct RngSmem {
    u64 *Bs;          // g's canonical keys
    uint16_t *cur;    // per row: first column not yet consumed
    uint16_t *ce;     // per row: the column edge at the current piece's end
    u64 *kA, *kB;     // sort buffers (raw product keys)
    uint16_t *iA, *iB;
    u64 *cv;          // product coefficients: word k of product q at cv[k * CHUNK + q]
    u32 *hist;        // bucket counts / offsets of the sort
};

// Per coefficient word count CW: the chunk, sort items per thread, products
// per lane of a piece and the shared-memory layout.  While a piece's
// products are generated, the sort's second key buffer (kB, free until the
// scatter) holds the piece's compacted row tables: the c-th row with
// products is crow[c] and its products start at coff[c] (coff[nnz] = O),
// u16 arrays at offsets 0 and CROW.  The scan of the packed per-thread
// counts (products in the low word, rows with products in the high word)
// gives each thread's starts; rng_piece's first barrier publishes them.
template <u32 CW, u32 MAXT>
struct Rng {
    // threads: 1024 where the shared memory has room for the radix
    // fallback's per-warp histograms (operands of at most 4096 terms), else
    // 512; one CTA per SM either way
    static constexpr int T = MAXT <= 4096 ? 1024 : 512;
    static constexpr u32 W = T / 32;
    static constexpr u32 CHUNK = rng_chunk(CW);
    static constexpr int IPT = CHUNK / T;
    static constexpr u32 LANE_MAX = (CHUNK / W + 31) / 32;  // products per lane of a piece
    static constexpr u32 CROW = CHUNK + 8;
    static constexpr u32 HIST_WORDS = (T / 32) * 256 > BUCKETS ? (T / 32) * 256 : BUCKETS;
    static constexpr size_t SMEM = (size_t)MAXT * 8 + MAXT * 2 * 2 +
                                   (size_t)CHUNK * (8 + 8 + 2 + 2 + 8 * CW) + (size_t)HIST_WORDS * 4;
    static_assert((CROW + CHUNK) * 2 <= CHUNK * 8, "row tables overflow the second key buffer");
    static_assert(CHUNK <= 65535 && CHUNK % T == 0, "16-bit product offsets, whole sort items per thread");

    static __device__ __forceinline__ RngSmem carve(unsigned char *p)
    {
        RngSmem m;
        m.Bs = (u64 *)p;
        m.kA = m.Bs + MAXT;
        m.kB = m.kA + CHUNK;
        m.cv = m.kB + CHUNK;
        m.hist = (u32 *)(m.cv + CW * CHUNK);
        m.cur = (uint16_t *)(m.hist + HIST_WORDS);
        m.iA = m.cur + MAXT;
        m.iB = m.iA + CHUNK;
        m.ce = m.iB + CHUNK;
        return m;
    }
};

__device__ __forceinline__ u64 row_counts(u32 cnt) { return (u64)cnt | ((u64)(cnt != 0) << 32); }

// The piece's row tables (in kB), and the sort's bucket counts cleared for
// the generation to fill.  Runs between the caller's scan and rng_piece's
// first barrier; the previous piece no longer reads kB or hist by then.
template <u32 CW, u32 MAXT>
__device__ __forceinline__ void piece_offsets(RngSmem &m, u32 cf, u64 base, u64 total)
{
    typedef Rng<CW, MAXT> R;
    uint16_t *coff = (uint16_t *)m.kB, *crow = coff + R::CROW;
    u32 pb = (u32)base, cb = (u32)(base >> 32);
    for (u32 r = threadIdx.x; r < cf; r += R::T) {
        const u32 cnt = (u32)m.ce[r] - m.cur[r];
        if (cnt) {
            coff[cb] = (uint16_t)pb;
            crow[cb] = (uint16_t)r;
            cb++;
            pb += cnt;
        }
    }
    if (threadIdx.x == 0) coff[total >> 32] = (uint16_t)total;
    for (u32 x = threadIdx.x; x < BUCKETS; x += R::T) m.hist[x] = 0;
}

// Sorts the piece's n (key, index) pairs in kA/iA by key, the bucket counts
// having been taken while the products were generated (bucket = the top 12
// significant bits of key - lo, clamped; with shift 0 one key value per
// bucket).  Each pair moves once by bucket and once to its place inside the
// bucket, found by counting the bucket's smaller keys (ties by position);
// with shift 0 the scatter alone sorts.  Equal keys come out adjacent in no
// particular order.  A bucket with more than BUCKET_RANK_MAX pairs sends the
// piece to the LSD radix sort instead.  On return m.kA/m.iA hold the sorted
// pairs (the buffers may have swapped).  All threads call; ends with a
// barrier.
template <u32 CW, u32 MAXT>
__device__ void sort_piece(RngSmem &m, u32 n, u64 lo, u64 span, int shift, u64 *ws)
{
    typedef Rng<CW, MAXT> R;
    constexpr u32 PER = BUCKETS / R::T;
    static_assert(BUCKETS % R::T == 0, "buckets per thread");
    __shared__ u32 s_bmax;
    const u32 tid = threadIdx.x;
    if (tid == 0) s_bmax = 0;
    // exclusive bucket offsets (thread t owns buckets [t PER, t PER + PER))
    u32 c[PER];
    u32 sum = 0, mx = 0;
#pragma unroll
    for (u32 q = 0; q < PER; q++) {
        c[q] = m.hist[tid * PER + q];
        sum += c[q];
        mx = c[q] > mx ? c[q] : mx;
    }
    u64 tot;
    u32 run = (u32)block_exclusive_scan(sum, tot, ws);  // its barriers order s_bmax = 0 first
    if (shift > 0 && mx > BUCKET_RANK_MAX) atomicMax(&s_bmax, mx);
#pragma unroll
    for (u32 q = 0; q < PER; q++) {
        m.hist[tid * PER + q] = run;
        run += c[q];
    }
    __syncthreads();
    if (s_bmax > BUCKET_RANK_MAX) {
        block_sort_pairs<R::T, R::IPT>(m.kA, m.iA, m.kB, m.iB, n, varying_bits(lo, lo + span), m.hist, ws);
        return;
    }
    // scatter by bucket; afterwards hist[b] is the end of bucket b
    if (shift > 0) {
        for (u32 q = tid; q < n; q += R::T) {
            const u64 key = m.kA[q];
            const u32 b = (u32)min((key - lo) >> shift, (u64)BUCKETS - 1);
            const u32 p = atomicAdd(&m.hist[b], 1u);
            m.kB[p] = key;
            m.iB[p] = m.iA[q];
        }
    } else {
        // one key value per bucket, often repeated: one atomic per distinct
        // bucket of a warp
        const u32 lane = tid & 31, nround = (n + 31u) & ~31u;
        for (u32 i = tid & ~31u; i < nround; i += R::T) {
            const u32 q = i + lane;
            const bool valid = q < n;
            const u64 key = valid ? m.kA[q] : 0;
            const u32 b = valid ? (u32)min(key - lo, (u64)BUCKETS - 1) : BUCKETS;
            const u32 peers = __match_any_sync(0xffffffffu, b);
            const u32 leader = (u32)(__ffs(peers) - 1);
            u32 base = 0;
            if (valid && lane == leader) base = atomicAdd(&m.hist[b], (u32)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (valid) {
                const u32 p = base + (u32)__popc(peers & ((1u << lane) - 1u));
                m.kB[p] = key;
                m.iB[p] = m.iA[q];
            }
        }
    }
    __syncthreads();
    if (shift == 0) {
        u64 *tk = m.kA;
        m.kA = m.kB;
        m.kB = tk;
        uint16_t *ti = m.iA;
        m.iA = m.iB;
        m.iB = ti;
        return;
    }
    // rank inside the bucket, written back to the A buffers
    for (u32 x = tid; x < n; x += R::T) {
        const u64 key = m.kB[x];
        const u32 b = (u32)min((key - lo) >> shift, (u64)BUCKETS - 1);
        const u32 beg = b ? m.hist[b - 1] : 0u, end = m.hist[b];
        u32 rank = 0;
        for (u32 y = beg; y < end; y++) {
            const u64 o = m.kB[y];
            rank += (o < key || (o == key && y < x)) ? 1u : 0u;
        }
        m.kA[beg + rank] = key;
        m.iA[beg + rank] = m.iB[x];
    }
    __syncthreads();
}

// One piece [plo, phi) whose column edges are cur (start) and ce (end),
// with tables from piece_offsets: generate its O <= CHUNK products, sort,
// reduce, and write the non-zero terms at claim_r + written,
// claim_r being the range's output base as thread 0 holds it.  Returns the
// terms written.  Ends without a barrier: the caller's next scan separates
// this piece's reads of the shared buffers from the next piece's writes.
// Where a range's terms go: the scratch (CW words per term) or, for a
// direct product, its output (the product's own words per term).
struct Dest {
    u64 *key, *coef;
    u32 words;
};

template <u32 CW, u32 MAXT>
__device__ u64 rng_piece(const BArgs &a, const BDesc &d, RngSmem &m, const u64 *A, const u64 *Ac, const u64 *Bc,
                         u64 total, u64 plo, u64 phi, u64 claim_r, u64 written, u64 *s_out, u64 *ws, Dest dst_)
{
    typedef Rng<CW, MAXT> R;
    const u32 tid = threadIdx.x;
    // a one-word batch holds mod-p products only
    const bool m61 = CW == 1 || (int)d.kind == PM_COEF_M61;
    const u32 O = (u32)total, nnz = (u32)(total >> 32);
    const uint16_t *coff = (const uint16_t *)m.kB, *crow = coff + R::CROW;
    // bucket of a key: the top 12 significant bits of key - plo
    const u64 span = phi - 1 - plo;
    const int shift = span >> 12 ? 52 - __clzll((long long)span) : 0;
    __syncthreads();
    // warp w takes a contiguous slice of the products, lanes interleaved so
    // that neighbouring lanes read neighbouring columns.  The warp first
    // finds the rows of all its products, then issues their loads together,
    // so the global-load latency is paid once per piece.
    const u32 lane = tid & 31, w = tid >> 5;
    {
        const u32 per_warp = ((O + R::W - 1) / R::W + 31u) & ~31u;
        const u32 p0 = w * per_warp, p1 = min(p0 + per_warp, O);
        u32 rr[R::LANE_MAX], jj[R::LANE_MAX];
        const u32 q0 = p0 + lane;
        if (p0 < p1) {
            // compacted row holding product p0 (last c with coff[c] <= p0),
            // by a 32-way search: each round every lane probes one point
            u32 ca = 0, n = nnz;
            while (n > 1) {
                const u32 step = (n + 31) >> 5;
                const bool le = lane * step < n && coff[ca + lane * step] <= p0;
                const u32 k = 31 - __clz(__ballot_sync(0xffffffffu, le));
                ca += k * step;
                n = min(step, n - k * step);
            }
            // 32 consecutive products [qa, qa + 32) touch at most 32 rows
            // past ca, and every row past ca starts at or after qa: lane L
            // looks at row ca + 1 + L, the rows starting inside the group
            // set one bit each, and a product's row is ca plus the bits at
            // or below its lane
#pragma unroll
            for (u32 t = 0; t < R::LANE_MAX; t++) {
                const u32 qa = p0 + 32 * t;
                if (qa < p1) {
                    const u32 c = ca + 1 + lane;
                    const u32 st = c < nnz ? (u32)coff[c] : 0xffffffffu;
                    const u32 bit = st - qa < 32u ? 1u << (st - qa) : 0u;
                    const u32 mask = __reduce_or_sync(0xffffffffu, bit);
                    const u32 cc = ca + (u32)__popc(mask & ((2u << lane) - 1u));
                    rr[t] = crow[cc];
                    jj[t] = m.cur[rr[t]] + (qa + lane - coff[cc]);
                    ca += (u32)__popc(mask);
                }
            }
#pragma unroll
            for (u32 t = 0; t < R::LANE_MAX; t++) {
                const u32 q = q0 + 32 * t;
                if (q < p1) {
                    const u32 r2 = rr[t], j = jj[t];
                    const u64 key = A[r2] + m.Bs[j];
                    m.kA[q] = key;
                    m.iA[q] = (uint16_t)q;
                    atomicAdd(&m.hist[(u32)min((key - plo) >> shift, (u64)BUCKETS - 1)], 1u);
                    if (m61) {
                        m.cv[q] = m61_reduce(m61_mul_lazy(Ac[r2], Bc[j]));
                    } else {
                        u64 lo2, hi2;
                        mul_i64_wide((i64)Ac[r2], (i64)Bc[j], lo2, hi2);
                        m.cv[q] = lo2;
                        m.cv[R::CHUNK + q] = hi2;
                    }
                }
            }
        }
    }
    __syncthreads();
    const u32 n = O;
    sort_piece<CW, MAXT>(m, n, plo, span, shift, ws);
    // segmented reduction: warp w owns the run heads in a contiguous
    // segment of the sorted pairs (a run may continue past it); positions
    // come from ballots and one block scan over the warps' counts
    const u32 seg = ((n + R::W - 1) / R::W + 31u) & ~31u;
    const u32 s0 = w * seg, s1 = min(s0 + seg, n);
    u64 v0[R::LANE_MAX], v1[R::LANE_MAX];
    u32 nzmask[R::LANE_MAX];
    u32 wcount = 0;
#pragma unroll
    for (u32 t = 0; t < R::LANE_MAX; t++) {
        const u32 i = s0 + 32 * t + lane;
        v0[t] = 0;
        v1[t] = 0;
        bool nz = false;
        if (i < s1 && (i == 0 || m.kA[i] != m.kA[i - 1])) {
            const u64 key = m.kA[i];
            for (u32 j = i; j < n && m.kA[j] == key; j++) {
                const u32 src = m.iA[j];
                if (m61) v0[t] = m61_add(v0[t], m.cv[src]);
                else add128(v0[t], v1[t], m.cv[src], m.cv[R::CHUNK + src]);
            }
            nz = (v0[t] | v1[t]) != 0;
        }
        nzmask[t] = __ballot_sync(0xffffffffu, nz);
        wcount += (u32)__popc(nzmask[t]);
    }
    // thread 0 publishes the output base here, so the claim's atomic
    // (issued before the piece was generated) is waited for only now; the
    // scan's barriers make it visible
    if (tid == 0) *s_out = claim_r + written;
    u64 nout;
    u64 wbase = block_exclusive_scan(lane == 0 ? wcount : 0u, nout, ws);
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    const u64 out = *s_out;
    u32 before = 0;
#pragma unroll
    for (u32 t = 0; t < R::LANE_MAX; t++) {
        const u32 i = s0 + 32 * t + lane;
        if ((nzmask[t] >> lane) & 1u) {
            const u64 dst = out + wbase + before + (u32)__popc(nzmask[t] & ((1u << lane) - 1u));
            dst_.key[dst] = m.kA[i];
            dst_.coef[dst_.words * dst] = v0[t];
            if (dst_.words == 2) dst_.coef[2 * dst + 1] = v1[t];
        }
        before += (u32)__popc(nzmask[t]);
    }
    return nout;
}

// sum of all products of a single-monomial piece with more than CHUNK
// products; writes at most one term
template <u32 CW, u32 MAXT>
__device__ u64 rng_single(const BArgs &a, const BDesc &d, RngSmem &m, const u64 *A, const u64 *Ac, const u64 *Bc,
                          u32 cf, u64 key, u64 out, u64 *ws, Dest dst_)
{
    typedef Rng<CW, MAXT> R;
    const bool m61 = CW == 1 || (int)d.kind == PM_COEF_M61;
    u64 s0 = 0, s1 = 0;
    for (u32 r = threadIdx.x; r < cf; r += R::T)
        for (u32 j = m.cur[r]; j < m.ce[r]; j++) {
            if (m61) {
                s0 = m61_add(s0, m61_reduce(m61_mul_lazy(Ac[r], Bc[j])));
            } else {
                u64 lo, hi;
                mul_i64_wide((i64)Ac[r], (i64)Bc[j], lo, hi);
                add128(s0, s1, lo, hi);
            }
        }
    // block reduction through the scan helper, word by word with carries
    __shared__ u64 red[2 * (R::T / 32)];
    const u32 lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
        const u64 o0 = __shfl_down_sync(0xffffffffu, s0, dd), o1 = __shfl_down_sync(0xffffffffu, s1, dd);
        if (m61) s0 = m61_add(s0, o0);
        else add128(s0, s1, o0, o1);
    }
    if (lane == 0) {
        red[2 * w] = s0;
        red[2 * w + 1] = s1;
    }
    __syncthreads();
    __shared__ u64 wrote;
    if (threadIdx.x == 0) {
        u64 r0w = 0, r1w = 0;
        for (int ww = 0; ww < R::T / 32; ww++) {
            if (m61) r0w = m61_add(r0w, red[2 * ww]);
            else add128(r0w, r1w, red[2 * ww], red[2 * ww + 1]);
        }
        wrote = 0;
        if ((r0w | r1w) != 0) {
            dst_.key[out] = key;
            dst_.coef[dst_.words * out] = r0w;
            if (dst_.words == 2) dst_.coef[2 * out + 1] = r1w;
            wrote = 1;
        }
    }
    __syncthreads();
    return wrote;
}

template <u32 CW, u32 MAXT>
__global__ void __launch_bounds__(Rng<CW, MAXT>::T, 1) kb_ranges(BArgs a)
{
    typedef Rng<CW, MAXT> R;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    __shared__ u32 item;
    __shared__ u64 claim;
    RngSmem m = R::carve(smem);
    const u32 tid = threadIdx.x;
    for (;;) {
        if (tid == 0) item = atomicAdd(a.work, 1u);
        __syncthreads();
        const u32 it = item;
        __syncthreads();
        if (it >= a.nitems) break;
        const u32 p = a.item_prod[it], first = a.item_first[it];
        const BDesc &d = a.D[p];
        if (d.status || first >= d.nranges) continue;
        const u32 last = min(first + a.per_item, d.nranges);
        // rows run over the smaller operand (the product is commutative), so
        // each range visits as few rows as possible
        const bool swap = d.cf > d.cg;
        const u32 cf = swap ? d.cg : d.cf, cg = swap ? d.cf : d.cg;
        const u64 *Fk = a.ck + d.op_off, *Fc = a.cc + d.op_off;
        const u64 *Gk = Fk + d.nf, *Gc = Fc + d.nf;
        const u64 *A = swap ? Gk : Fk, *Ac = swap ? Gc : Fc;
        const u64 *Bg = swap ? Fk : Gk, *Bc = swap ? Fc : Gc;
        // g's keys in shared memory when they fit, else read through L1
        m.Bs = (u64 *)smem;
        if (cg <= MAXT) {
            for (u32 j = tid; j < cg; j += R::T) m.Bs[j] = Bg[j];
        } else {
            m.Bs = const_cast<u64 *>(Bg);
        }
        __syncthreads();
        // rows of this thread: tid, tid + R::T, ... (neighbouring lanes on
        // neighbouring rows: coalesced row loads, conflict-free cursors); a
        // piece's compacted row table lists them thread by thread, which the
        // generation and the sort do not mind.  Cursors at the first range's
        // start.
        {
            const u64 lo = a.rlo[d.rg_off + first];
            for (u32 r = tid; r < cf; r += R::T) {
                const u64 ar = A[r];
                u32 c = 0;
                if (lo > ar) {
                    const u64 x = lo - ar;
                    u32 lo2 = 0, len = cg;
                    while (len > 0) {
                        const u32 half = len >> 1;
                        if (m.Bs[lo2 + half] < x) {
                            lo2 += half + 1;
                            len -= half + 1;
                        } else {
                            len = half;
                        }
                    }
                    c = lo2;
                }
                m.cur[r] = (uint16_t)c;
            }
        }
        // a direct product's terms below the first range: the sum of the
        // row cursors (term products with keys below the range's start)
        const Dest dst_ = d.direct ? Dest{d.hkey, d.hcoef, (int)d.kind == PM_COEF_M61 ? 1u : 2u}
                                   : Dest{a.skey, a.scoef, CW};
        u64 omega = 0;
        if (d.direct) {
            u64 mine_c = 0;
            for (u32 r = tid; r < cf; r += R::T) mine_c += m.cur[r];
            block_exclusive_scan(mine_c, omega, ws);
        }
        __syncthreads();
        for (u32 k = first; k < last; k++) {
            const u64 rlo_k = a.rlo[d.rg_off + k], rhi_k = a.rhi[d.rg_off + k];
            // edges at the range end and the range's product count
            u64 mine = 0;
            for (u32 r = tid; r < cf; r += R::T) {
                const u64 ar = A[r];
                const u32 e = rhi_k > ar ? gallop_up(m.Bs, cg, m.cur[r], rhi_k - ar) : m.cur[r];
                m.ce[r] = (uint16_t)e;
                mine += row_counts(e - m.cur[r]);
            }
            u64 tot;
            const u64 base = block_exclusive_scan(mine, tot, ws);
            const u64 O = (u32)tot;
            // the range's output base: a direct product's term products
            // below the range; otherwise claimed scratch (at most O terms),
            // held by thread 0 only and waited for when a piece publishes it
            u64 claim_r = omega;
            if (!d.direct && tid == 0) claim_r = atomicAdd(a.bump, O);
            omega += O;
            u64 written = 0;
            if (O <= R::CHUNK) {
                if (O) {
                    piece_offsets<CW, MAXT>(m, cf, base, tot);
                    written = rng_piece<CW, MAXT>(a, d, m, A, Ac, Bc, tot, rlo_k, rhi_k, claim_r, 0, &claim, ws, dst_);
                }
                // own rows only: other threads read these cursors after the
                // next scan
                for (u32 r = tid; r < cf; r += R::T) m.cur[r] = m.ce[r];
            } else {
                // bisect by key: pieces [plo, phi) with at most CHUNK
                // products, or a single monomial
                u64 plo = rlo_k;
                while (plo < rhi_k) {
                    u64 phi = rhi_k;
                    for (;;) {
                        u64 cnt_mine = 0;
                        for (u32 r = tid; r < cf; r += R::T) {
                            const u64 ar = A[r];
                            const u32 e = phi > ar ? gallop_up(m.Bs, cg, m.cur[r], phi - ar) : m.cur[r];
                            m.ce[r] = (uint16_t)e;
                            cnt_mine += row_counts(e - m.cur[r]);
                        }
                        u64 ptot;
                        const u64 pbase = block_exclusive_scan(cnt_mine, ptot, ws);
                        const u64 PO = (u32)ptot;
                        if (PO <= R::CHUNK) {
                            if (PO) {
                                piece_offsets<CW, MAXT>(m, cf, pbase, ptot);
                                written += rng_piece<CW, MAXT>(a, d, m, A, Ac, Bc, ptot, plo, phi, claim_r, written, &claim, ws,
                                                               dst_);
                            }
                            break;
                        }
                        if (phi - plo == 1) {
                            written += rng_single<CW, MAXT>(a, d, m, A, Ac, Bc, cf, plo, claim_r + written, ws, dst_);
                            break;
                        }
                        phi = plo + (phi - plo) / 2;
                    }
                    for (u32 r = tid; r < cf; r += R::T) m.cur[r] = m.ce[r];
                    plo = phi;
                }
            }
            if (tid == 0) {
                a.rbase[d.rg_off + k] = claim_r;
                a.rcount[d.rg_off + k] = written;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// B4: concatenate each product's ranges into its output
//   B4a (one CTA per product): sizes, capacity check, and per range its
//       place in the output -- written over the range's bounds, which B3
//       no longer needs: rlo = destination offset, rhi = product index (or
//       SKIP for a range slot that is not copied);
//   B4b (all SMs): warps copy ranges, so one large product's copy is
//       spread over the whole GPU.
// ---------------------------------------------------------------------------

constexpr u64 SKIP = ~0ull;

// Compaction units of direct products whose ranges hold fewer terms than
// term products (some products shared a monomial): unit u covers the
// output positions [u CMP_CH, (u + 1) CMP_CH), each taken from its range's
// place Omega_k + (x - F_k) >= x.  A unit reads all its terms, publishes
// that in its flag, waits for the flags of the units whose sources lie in
// its destination (earlier units only: sources are never left of their
// destinations), then writes.
constexpr int CMP_T = 512;
constexpr u32 CMP_PER = 8;
constexpr u32 CMP_CH = CMP_T * CMP_PER;

__global__ void __launch_bounds__(FIN_T) kb_finish(BArgs a)
{
    __shared__ u64 ws[32];
    const u32 p = blockIdx.x, tid = threadIdx.x;
    BDesc &d = a.D[p];
    const u32 nr = d.status ? 0u : d.nranges;
    u64 *rlo = a.rlo + d.rg_off, *rhi = a.rhi + d.rg_off;
    const u64 *rc = a.rcount + d.rg_off;
    u64 total = 0;
    for (u32 k0 = 0; k0 < nr; k0 += FIN_T) {
        const u32 k = k0 + tid;
        u64 cnt;
        block_exclusive_scan(k < nr ? rc[k] : 0, cnt, ws);
        total += cnt;
    }
    if (d.direct) {
        // the terms are in h already; in place unless monomials repeated,
        // else the ranges' destinations (rlo) and the compaction units
        __shared__ u64 s_base;
        const bool moves = nr && total != (u64)d.cf * d.cg;
        u64 run = 0;
        for (u32 k0 = 0; k0 < d.rcap; k0 += FIN_T) {
            const u32 k = k0 + tid;
            u64 cnt;
            const u64 at = run + block_exclusive_scan(k < nr ? rc[k] : 0, cnt, ws);
            if (k < d.rcap) {
                rlo[k] = moves && k < nr ? at : 0;
                rhi[k] = SKIP;
            }
            run += cnt;
        }
        const u64 units = moves ? (total + CMP_CH - 1) / CMP_CH : 0;
        if (tid == 0) {
            d.n_out = d.status ? 0 : total;
            s_base = units ? atomicAdd(&a.ucount[0], (u32)units) : 0;
            d.cmp_base = s_base;
        }
        __syncthreads();
        for (u64 i = tid; i < units; i += FIN_T) {
            a.uprod[s_base + i] = p;
            a.uflag[s_base + i] = 0;
        }
        return;
    }
    const bool fits = total <= d.hcap;
    u64 run = 0;
    for (u32 k0 = 0; k0 < d.rcap; k0 += FIN_T) {
        const u32 k = k0 + tid;
        u64 cnt;
        const u64 at = run + block_exclusive_scan(k < nr ? rc[k] : 0, cnt, ws);
        if (k < d.rcap) {
            const bool copy = fits && k < nr;
            rlo[k] = copy ? at : 0;
            rhi[k] = copy ? (u64)p : SKIP;
        }
        run += cnt;
    }
    if (tid == 0) {
        d.n_out = d.status ? 0 : total;
        if (!fits && !d.status) d.status |= ST_CAPACITY;
    }
}

__global__ void __launch_bounds__(256) kb_copy(BArgs a)
{
    const u32 lane = threadIdx.x & 31;
    const u64 warps = (u64)gridDim.x * (blockDim.x >> 5);
    for (u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < a.rg_total; r += warps) {
        const u64 p = a.rhi[r];
        if (p == SKIP) continue;
        const BDesc &d = a.D[p];
        const u64 src = a.rbase[r], dst = a.rlo[r], n = a.rcount[r];
        for (u64 t = lane; t < n; t += 32) {
            d.hkey[dst + t] = a.skey[src + t];
            if (d.kind == PM_COEF_M61) {
                d.hcoef[dst + t] = a.scoef[a.cw * (src + t)];
            } else {
                d.hcoef[2 * (dst + t)] = a.scoef[2 * (src + t)];
                d.hcoef[2 * (dst + t) + 1] = a.scoef[2 * (src + t) + 1];
            }
        }
    }
}

__device__ __forceinline__ u32 ld_acquire_u32(const u32 *p)
{
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(u32 *p, u32 v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// last k in [0, n) with v(k) <= x (v ascending, v(0) <= x), by one warp:
// each round the 32 lanes probe 32 evenly spaced points
template <class V>
__device__ __forceinline__ u32 warp_last_le(V v, u32 n, u64 x)
{
    const u32 lane = threadIdx.x & 31;
    u32 a0 = 0;
    while (n > 1) {
        const u32 step = (n + 31) >> 5;
        const bool le = lane * step < n && v(a0 + lane * step) <= x;
        const u32 k = 31 - __clz(__ballot_sync(0xffffffffu, le));
        a0 += k * step;
        n = min(step, n - k * step);
    }
    return a0;
}

// B4c (all SMs): the compaction units, taken in list order from a counter.
// A unit only waits for units listed before it, which were taken earlier by
// running CTAs and publish their reads without waiting, so every wait ends;
// a wait still bounded, past which the product fails with ST_INTERNAL.
__global__ void __launch_bounds__(CMP_T) kb_compact(BArgs a)
{
    __shared__ u32 s_g, s_fail;
    __shared__ u32 s_k0, s_ulo, s_ident;
    const u32 tid = threadIdx.x, lane = tid & 31;
    for (;;) {
        if (tid == 0) {
            s_g = atomicAdd(&a.ucount[1], 1u);
            s_fail = 0;
        }
        __syncthreads();
        const u32 g = s_g;
        if (g >= *(volatile u32 *)&a.ucount[0]) break;
        const u32 p = a.uprod[g];
        BDesc &d = a.D[p];
        const u32 nr = d.nranges;
        const u64 *F = a.rlo + d.rg_off, *Om = a.rbase + d.rg_off, *rc = a.rcount + d.rg_off;
        const u64 u = g - d.cmp_base, x0 = u * CMP_CH, x1 = min(x0 + CMP_CH, d.n_out);
        const u32 words = (int)d.kind == PM_COEF_M61 ? 1u : 2u;
        if (tid < 32) {
            auto Fv = [&](u32 k) { return F[k]; };
            auto Ev = [&](u32 k) { return Om[k] + rc[k]; };
            const u32 k0 = warp_last_le(Fv, nr, x0), k1 = warp_last_le(Fv, nr, x1 - 1);
            // the smallest destination whose source reaches x0 (range j, the
            // first whose sources end above x0): its unit is the first one
            // to wait for
            const u32 j = Ev(0) > x0 ? 0u : warp_last_le(Ev, nr, x0) + 1;
            if (lane == 0) {
                s_k0 = k0;
                // Omega_k - F_k never decreases with k: the unit stays in
                // place when its last range does
                s_ident = Om[k1] == F[k1];
                s_ulo = j < nr ? (u32)((F[j] + (x0 > Om[j] ? x0 - Om[j] : 0)) / CMP_CH) : (u32)u;
            }
        }
        __syncthreads();
        if (s_ident) {
            if (tid == 0) st_release_u32(&a.uflag[g], 1u);
            __syncthreads();
            continue;
        }
        // read: position x of range k (last k with F_k <= x) comes from
        // Omega_k + x - F_k
        u64 kk[CMP_PER], c0[CMP_PER], c1[CMP_PER];
        u32 k = s_k0;
#pragma unroll
        for (u32 q = 0; q < CMP_PER; q++) {
            const u64 x = x0 + q * CMP_T + tid;
            if (x < x1) {
                while (k + 1 < nr && F[k + 1] <= x) k++;
                const u64 src = Om[k] + (x - F[k]);
                kk[q] = d.hkey[src];
                c0[q] = d.hcoef[words * src];
                c1[q] = words == 2 ? d.hcoef[2 * src + 1] : 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release_u32(&a.uflag[g], 1u);
        }
        // wait for the earlier units whose sources this unit overwrites
        const u32 ulo = s_ulo;
        for (u32 w = ulo + tid; w < (u32)u; w += CMP_T) {
            const u32 *f = &a.uflag[d.cmp_base + w];
            u32 spins = 0;
            while (!ld_acquire_u32(f)) {
                if (++spins > (1u << 22)) {
                    atomicOr(&s_fail, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) atomicOr(&d.status, ST_INTERNAL);
        } else {
#pragma unroll
            for (u32 q = 0; q < CMP_PER; q++) {
                const u64 x = x0 + q * CMP_T + tid;
                if (x < x1) {
                    d.hkey[x] = kk[q];
                    d.hcoef[words * x] = c0[q];
                    if (words == 2) d.hcoef[2 * x + 1] = c1[q];
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host: layout, enqueue, plans (graph), workspace mode
// ---------------------------------------------------------------------------

template <class K>
static void set_smem_b(K kernel, size_t bytes)
{
    PM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

constexpr size_t CAN_SMEM = (size_t)BT_MAX_TERMS * (8 + 8 + 2 + 2) + (CAN_T / 32) * 256 * 4;
constexpr size_t PLAN_SMEM = (size_t)PLAN_SAMPLES * (8 + 8 + 2 + 2) + (PLAN_T / 32) * 256 * 4;

struct BatchSizes {
    u64 op_total = 0, rg_total = 0, prod_total = 0, term_total = 0;   // prod_total: scratch terms
    u64 unit_total = 0;           // compaction units the direct products may need
    u32 nitems = 0, cw = 1, maxt = 4096, target = 0, per_item = 0;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// device workspace layout (every region 256-byte aligned)
struct WsLayout {
    size_t D, ck, cc, rlo, rhi, rbase, rcount, ip, ifr, work, bump, skey, scoef, uprod, uflag, ucount, total;
    WsLayout(u32 count, const BatchSizes &z)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            size_t at = o;
            o += align256(bytes ? bytes : 8);
            return at;
        };
        D = take(sizeof(BDesc) * count);
        ck = take(8 * (z.op_total + 1));
        cc = take(8 * (z.op_total + 1));
        rlo = take(8 * z.rg_total);
        rhi = take(8 * z.rg_total);
        rbase = take(8 * z.rg_total);
        rcount = take(8 * z.rg_total);
        ip = take(4 * (size_t)z.nitems);
        ifr = take(4 * (size_t)z.nitems);
        work = take(8);
        bump = take(8);
        skey = take(8 * (z.prod_total + 1));
        scoef = take(8 * (size_t)z.cw * (z.prod_total + 1));
        uprod = take(4 * z.unit_total);
        uflag = take(4 * z.unit_total);
        ucount = take(8);
        total = o;
    }
};

// host staging layout: descriptors, then the two work-item tables
static size_t stage_bytes(u32 count, const BatchSizes &z)
{
    return sizeof(BDesc) * count + 8 * (size_t)z.nitems;
}

// Validate the items; with descs/ip/ifr non-null also write the descriptors
// and the work-item tables.
static BatchSizes build_batch(const pm_batch_item *items, u32 count, const pm_batch_options *opt, BDesc *descs,
                              u32 *ip, u32 *ifr)
{
    if (!items || count == 0) throw Error(PM_EINVAL, "empty batch");
    pm_batch_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    BatchSizes z;
    // the coefficient words, hence the chunk and the default target
    for (u32 p = 0; p < count; p++)
        if (items[p].coef_kind == PM_COEF_I64_ACC128) z.cw = 2;
    z.target = o.range_target ? o.range_target : rng_target_default(z.cw);
    z.per_item = o.ranges_per_item ? o.ranges_per_item : 16;
    if (z.target < 64 || z.target > rng_chunk(z.cw) || z.per_item < 1 || z.per_item > 4096)
        throw Error(PM_EINVAL, "bad batch options");
    for (u32 p = 0; p < count; p++) {
        const pm_batch_item &it = items[p];
        const pm_packing &pk = it.pk;
        if (pk.nvars < 1 || pk.nvars > PM_MAX_VARS) throw Error(PM_EINVAL, "bad nvars");
        if (it.coef_kind != PM_COEF_M61 && it.coef_kind != PM_COEF_I64_ACC128) throw Error(PM_EINVAL, "bad kind");
        if (it.f.n > BT_MAX_TERMS || it.g.n > BT_MAX_TERMS) throw Error(PM_EINVAL, "operand above PM_BATCH_MAX_TERMS");
        if (it.f.n > 4096 || it.g.n > 4096) z.maxt = BT_MAX_TERMS;
        if ((it.f.n && (!it.f.exps || !it.f.coefs)) || (it.g.n && (!it.g.exps || !it.g.coefs)))
            throw Error(PM_EINVAL, "null operand arrays");
        if (it.h.cap && (!it.h.keys || !it.h.coefs)) throw Error(PM_EINVAL, "null output arrays");
        BDesc d;
        memset(&d, 0, sizeof(d));
        d.L.nv = pk.nvars;
        u32 sbits = 0;
        for (int v = (int)pk.nvars - 1; v >= 0; v--) {
            if (pk.field_bits[v] < 1 || pk.field_bits[v] > 32) throw Error(PM_EINVAL, "bad field width");
            d.L.off[v] = sbits;
            d.L.width[v] = pk.field_bits[v];
            sbits += pk.field_bits[v];
        }
        if (sbits > 64) throw Error(PM_EINVAL, "fields exceed 64 bits");
        d.kind = it.coef_kind;
        d.fe = it.f.exps;
        d.fc = (const u64 *)it.f.coefs;
        d.nf = (u32)it.f.n;
        d.ge = it.g.exps;
        d.gc = (const u64 *)it.g.coefs;
        d.ng = (u32)it.g.n;
        d.hkey = (u64 *)it.h.keys;
        d.hcoef = (u64 *)it.h.coefs;
        d.hcap = it.h.cap;
        d.op_off = z.op_total;
        z.op_total += d.nf + d.ng;
        const u64 P = (u64)d.nf * d.ng;
        // the output holds every term product: the range kernel writes the
        // results straight into it, no scratch
        d.direct = it.h.cap >= P ? 1u : 0u;
        if (!d.direct) z.prod_total += P;
        else z.unit_total += (P + CMP_CH - 1) / CMP_CH;
        z.term_total += P;
        u64 rcap = P ? (P + z.target - 1) / z.target + 1 : 1;
        if (rcap > PLAN_SAMPLES) rcap = PLAN_SAMPLES;
        d.rcap = (u32)rcap;
        d.rg_off = z.rg_total;
        z.rg_total += rcap;
        for (u32 f0 = 0; f0 < rcap; f0 += z.per_item) {
            if (ip) {
                ip[z.nitems] = p;
                ifr[z.nitems] = f0;
            }
            z.nitems++;
        }
        if (descs) descs[p] = d;
    }
    return z;
}

static BArgs carve_ws(unsigned char *base, u32 count, const BatchSizes &z)
{
    WsLayout w(count, z);
    BArgs a;
    memset(&a, 0, sizeof(a));
    a.D = (BDesc *)(base + w.D);
    a.count = count;
    a.ck = (u64 *)(base + w.ck);
    a.cc = (u64 *)(base + w.cc);
    a.rlo = (u64 *)(base + w.rlo);
    a.rhi = (u64 *)(base + w.rhi);
    a.rbase = (u64 *)(base + w.rbase);
    a.rcount = (u64 *)(base + w.rcount);
    a.item_prod = (const u32 *)(base + w.ip);
    a.item_first = (const u32 *)(base + w.ifr);
    a.nitems = z.nitems;
    a.work = (u32 *)(base + w.work);
    a.bump = (u64 *)(base + w.bump);
    a.skey = (u64 *)(base + w.skey);
    a.scoef = (u64 *)(base + w.scoef);
    a.cw = z.cw;
    a.maxt = z.maxt;
    a.target = z.target;
    a.per_item = z.per_item;
    a.rg_total = z.rg_total;
    a.uprod = (u32 *)(base + w.uprod);
    a.uflag = (u32 *)(base + w.uflag);
    a.ucount = (u32 *)(base + w.ucount);
    return a;
}

// The range kernel's shared memory, and the smallest carve-out that holds
// it, so that the rest of the SM's 256 KB stays L1 for the operand loads.
template <u32 CW, u32 MAXT>
static void set_ranges_smem()
{
    constexpr size_t bytes = Rng<CW, MAXT>::SMEM;
    set_smem_b(kb_ranges<CW, MAXT>, bytes);
    int dev = 0, per_sm = 0;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    if (per_sm <= 0) return;
    // dynamic + static shared memory + the 1 KB the system reserves per block
    cudaFuncAttributes fa;
    PM_CUDA(cudaFuncGetAttributes(&fa, kb_ranges<CW, MAXT>));
    const size_t need = bytes + fa.sharedSizeBytes + 1024;
    int pct = (int)((need * 100 + (size_t)per_sm - 1) / (size_t)per_sm);
    if (pct > 100) pct = 100;
    PM_CUDA(cudaFuncSetAttribute(kb_ranges<CW, MAXT>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
}

static void set_batch_smem()
{
    set_smem_b(kb_canon, CAN_SMEM);
    set_smem_b(kb_plan, PLAN_SMEM);
    set_ranges_smem<1, 4096>();
    set_ranges_smem<2, 4096>();
    set_ranges_smem<1, BT_MAX_TERMS>();
    set_ranges_smem<2, BT_MAX_TERMS>();
}

template <u32 CW, u32 MAXT>
static void launch_ranges(const BArgs &a, int sm_count, cudaStream_t s)
{
    kb_ranges<CW, MAXT><<<sm_count, Rng<CW, MAXT>::T, Rng<CW, MAXT>::SMEM, s>>>(a);
}

// the six kernels of the pass (counters cleared first)
static void launch_pass(const BArgs &a, int sm_count, cudaStream_t s)
{
    PM_CUDA(cudaMemsetAsync(a.work, 0, sizeof(u32), s));
    PM_CUDA(cudaMemsetAsync(a.bump, 0, sizeof(u64), s));
    PM_CUDA(cudaMemsetAsync(a.ucount, 0, 2 * sizeof(u32), s));
    kb_canon<<<2 * a.count, CAN_T, CAN_SMEM, s>>>(a);
    PM_CUDA(cudaGetLastError());
    kb_plan<<<a.count, PLAN_T, PLAN_SMEM, s>>>(a);
    PM_CUDA(cudaGetLastError());
    // operands of at most 4096 terms leave room for a larger L1
    if (a.maxt <= 4096) {
        if (a.cw == 1) launch_ranges<1, 4096>(a, sm_count, s);
        else launch_ranges<2, 4096>(a, sm_count, s);
    } else {
        if (a.cw == 1) launch_ranges<1, BT_MAX_TERMS>(a, sm_count, s);
        else launch_ranges<2, BT_MAX_TERMS>(a, sm_count, s);
    }
    PM_CUDA(cudaGetLastError());
    kb_finish<<<a.count, FIN_T, 0, s>>>(a);
    PM_CUDA(cudaGetLastError());
    kb_copy<<<sm_count * 8, 256, 0, s>>>(a);
    PM_CUDA(cudaGetLastError());
    kb_compact<<<sm_count * 2, CMP_T, 0, s>>>(a);
    PM_CUDA(cudaGetLastError());
}

static int item_code(u32 status)
{
    if (status & ST_EXP_OVERFLOW) return PM_EEXP_OVERFLOW;
    if (status & ST_COEF_BOUND) return PM_ECOEF_BOUND;
    if (status & ST_CAPACITY) return PM_ECAPACITY;
    if (status) return PM_ECUDA;
    return PM_OK;
}

// write statuses and sizes from result descriptors; returns the first error
static int collect(const BDesc *descs, u32 count, pm_batch_item *items, uint64_t *n_out, uint64_t *ranges)
{
    int worst = PM_OK;
    u64 no = 0, nr = 0;
    for (u32 p = 0; p < count; p++) {
        const int rc = item_code(descs[p].status);
        if (items) {
            items[p].status = rc;
            items[p].h.n = (rc == PM_OK || rc == PM_ECAPACITY) ? descs[p].n_out : 0;
        }
        if (rc == PM_OK) no += descs[p].n_out;
        nr += descs[p].nranges;
        if (rc != PM_OK && worst == PM_OK) worst = rc;
    }
    if (n_out) *n_out = no;
    if (ranges) *ranges = nr;
    return worst;
}

static int device_sms()
{
    int dev = 0, sms = 0;
    PM_CUDA(cudaGetDevice(&dev));
    PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

}  // namespace pm

struct pm_batch_plan {
    uint32_t count = 0;
    pm::BArgs args;
    pm::BatchSizes sizes;
    std::vector<pm::BDesc> h_desc;
    void *dws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    pm_batch_stats stats;
};

namespace pm {

static void batch_create(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                         pm_batch_plan *pl, cudaStream_t stream)
{
    BatchSizes z = build_batch(items, count, opt, nullptr, nullptr, nullptr);
    pl->count = count;
    pl->sizes = z;
    pl->h_desc.resize(count);
    std::vector<u32> ip(z.nitems), ifr(z.nitems);
    build_batch(items, count, opt, pl->h_desc.data(), ip.data(), ifr.data());
    WsLayout w(count, z);
    if (cudaMalloc(&pl->dws, w.total) != cudaSuccess) {
        cudaGetLastError();
        pl->dws = nullptr;
        throw Error(PM_ENOMEM, "batch plan allocation failed");
    }
    unsigned char *base = (unsigned char *)pl->dws;
    pl->args = carve_ws(base, count, z);
    PM_CUDA(cudaMemcpyAsync(base + w.D, pl->h_desc.data(), sizeof(BDesc) * count, cudaMemcpyHostToDevice, stream));
    PM_CUDA(cudaMemcpyAsync(base + w.ip, ip.data(), 4 * (size_t)z.nitems, cudaMemcpyHostToDevice, stream));
    PM_CUDA(cudaMemcpyAsync(base + w.ifr, ifr.data(), 4 * (size_t)z.nitems, cudaMemcpyHostToDevice, stream));
    PM_CUDA(cudaStreamSynchronize(stream));
    memset(&pl->stats, 0, sizeof(pl->stats));
    pl->stats.term_products = z.term_total;
    pl->stats.work_items = z.nitems;
    pl->stats.kernel_launches = 6;
    set_batch_smem();
    const int sms = device_sms();
    // capture the whole pass once; runs replay it
    cudaStream_t cs;
    PM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        try {
            launch_pass(pl->args, sms, cs);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            throw;
        }
        e = cudaStreamEndCapture(cs, &pl->graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) throw Error(PM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    PM_CUDA(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    pl->stats.graph = 1;
}

static void batch_destroy(pm_batch_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->dws) cudaFree(pl->dws);
    pl->exec = nullptr;
    pl->graph = nullptr;
    pl->dws = nullptr;
}

static int batch_finish(pm_batch_plan *pl, pm_batch_item *items, pm_batch_stats *st, cudaStream_t s)
{
    PM_CUDA(cudaMemcpyAsync(pl->h_desc.data(), pl->args.D, sizeof(BDesc) * pl->count, cudaMemcpyDeviceToHost, s));
    PM_CUDA(cudaStreamSynchronize(s));
    const int worst = collect(pl->h_desc.data(), pl->count, items, &pl->stats.n_out, &pl->stats.n_ranges);
    if (st) *st = pl->stats;
    return worst;
}

// workspace mode: everything stream-ordered, nothing allocated
void batch_enqueue_ws(const pm_batch_item *items, u32 count, const pm_batch_options *opt, void *dws, u64 dbytes,
                      void *hws, u64 hbytes, int sm_count, cudaStream_t s)
{
    const BatchSizes z = build_batch(items, count, opt, nullptr, nullptr, nullptr);
    const WsLayout w(count, z);
    if (!dws || dbytes < w.total || !hws || hbytes < stage_bytes(count, z))
        throw Error(PM_EINVAL, "batch workspace too small");
    if ((uintptr_t)dws & 255) throw Error(PM_EINVAL, "device workspace must be 256-byte aligned");
    unsigned char *h = (unsigned char *)hws, *base = (unsigned char *)dws;
    BDesc *descs = (BDesc *)h;
    u32 *ip = (u32 *)(h + sizeof(BDesc) * count), *ifr = ip + z.nitems;
    build_batch(items, count, opt, descs, ip, ifr);
    const BArgs a = carve_ws(base, count, z);
    PM_CUDA(cudaMemcpyAsync(base + w.D, descs, sizeof(BDesc) * count, cudaMemcpyHostToDevice, s));
    PM_CUDA(cudaMemcpyAsync(base + w.ip, ip, 4 * (size_t)z.nitems, cudaMemcpyHostToDevice, s));
    PM_CUDA(cudaMemcpyAsync(base + w.ifr, ifr, 4 * (size_t)z.nitems, cudaMemcpyHostToDevice, s));
    launch_pass(a, sm_count, s);
    PM_CUDA(cudaMemcpyAsync(descs, base + w.D, sizeof(BDesc) * count, cudaMemcpyDeviceToHost, s));
}

void batch_ws_sizes(const pm_batch_item *items, u32 count, const pm_batch_options *opt, u64 *dbytes, u64 *hbytes)
{
    const BatchSizes z = build_batch(items, count, opt, nullptr, nullptr, nullptr);
    const WsLayout w(count, z);
    *dbytes = w.total;
    *hbytes = stage_bytes(count, z);
}

int batch_collect_ws(pm_batch_item *items, u32 count, const void *hws)
{
    return collect((const BDesc *)hws, count, items, nullptr, nullptr);
}

void batch_prepare_device() { set_batch_smem(); }

u32 batch_range_chunk(u32 cw) { return rng_chunk(cw); }

}  // namespace pm

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------

template <class F>
static int bguard(F &&fn)
{
    try {
        return fn();
    } catch (const pm::Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return PM_ENOMEM;
    } catch (...) {
        return PM_ECUDA;
    }
}

extern "C" int pm_batch_plan_create(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                                    pm_batch_plan **plan, void *stream)
{
    if (!plan) return PM_EINVAL;
    *plan = nullptr;
    pm_batch_plan *pl = new (std::nothrow) pm_batch_plan();
    if (!pl) return PM_ENOMEM;
    int rc = bguard([&] {
        pm::batch_create(items, count, opt, pl, (cudaStream_t)stream);
        return PM_OK;
    });
    if (rc != PM_OK) {
        pm::batch_destroy(pl);
        delete pl;
        return rc;
    }
    *plan = pl;
    return PM_OK;
}

extern "C" int pm_batch_plan_run(pm_batch_plan *plan, void *stream)
{
    if (!plan || !plan->exec) return PM_EINVAL;
    return bguard([&] {
        PM_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
        return PM_OK;
    });
}

extern "C" int pm_batch_plan_finish(pm_batch_plan *plan, pm_batch_item *items, pm_batch_stats *stats, void *stream)
{
    if (!plan) return PM_EINVAL;
    return bguard([&] { return pm::batch_finish(plan, items, stats, (cudaStream_t)stream); });
}

extern "C" void pm_batch_plan_destroy(pm_batch_plan *plan)
{
    if (!plan) return;
    pm::batch_destroy(plan);
    delete plan;
}

extern "C" int pm_batch_polymul(pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                                pm_batch_stats *stats, void *stream)
{
    pm_batch_plan *pl = nullptr;
    int rc = pm_batch_plan_create(items, count, opt, &pl, stream);
    if (rc != PM_OK) return rc;
    rc = pm_batch_plan_run(pl, stream);
    if (rc == PM_OK) rc = pm_batch_plan_finish(pl, items, stats, stream);
    pm_batch_plan_destroy(pl);
    return rc;
}

extern "C" int pm_batch_workspace(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                                  uint64_t *device_bytes, uint64_t *host_bytes)
{
    if (!device_bytes || !host_bytes) return PM_EINVAL;
    return bguard([&] {
        pm::batch_ws_sizes(items, count, opt, (pm::u64 *)device_bytes, (pm::u64 *)host_bytes);
        return PM_OK;
    });
}

extern "C" int pm_batch_enqueue(const pm_batch_item *items, uint32_t count, const pm_batch_options *opt,
                                void *device_ws, uint64_t device_bytes, void *host_ws, uint64_t host_bytes,
                                void *stream)
{
    return bguard([&] {
        static std::once_flag once;
        std::call_once(once, [] { pm::batch_prepare_device(); });
        int dev = 0, sms = 0;
        PM_CUDA(cudaGetDevice(&dev));
        PM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        pm::batch_enqueue_ws(items, count, opt, device_ws, device_bytes, host_ws, host_bytes, sms,
                             (cudaStream_t)stream);
        return PM_OK;
    });
}

extern "C" int pm_batch_collect(pm_batch_item *items, uint32_t count, const void *host_ws)
{
    if (!items || !host_ws) return PM_EINVAL;
    return pm::batch_collect_ws(items, count, host_ws);
}
