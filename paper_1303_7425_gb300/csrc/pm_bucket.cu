// K-c + K-d for sparse products whose result is about as large as their
// term-product count (PM_STRATEGY_BUCKET): the pp-matrix is walked twice and
// every term product lands in a bucket of the output key space, then each
// bucket is sorted and reduced in shared memory -- the MergeSort of Alg. 1
// done as a most-significant-digit bucket pass followed by per-bucket sorts.
//
// The sort strategy (pm_range.cu) finds, for every output range, the column
// bounds of every row of the pp-matrix (FindEdge, Sec. 2): O(rows log n_g)
// per range, which dominates when a range of a few thousand products draws
// them from tens of thousands of rows.  Here a row's columns are read once
// per pass and each product finds its bucket by a table lookup:
//   0. bucket boundaries: the Sec. 5 grid over the operands, about eight
//      points per bucket, sorted; every eighth point bounds a bucket, so a
//      bucket holds about as many term products as the grid says eight
//      points stand for (the grid samples the pp-matrix evenly); a table
//      over the top bits of key - lo gives each cell's first bucket, and a
//      short binary search inside the cell finds the product's;
//   1. count: each bucket gets one count per product (a warp takes a row;
//      lanes run over consecutive columns, whose keys ascend, so lanes with
//      the same bucket add their run with one atomic);
//   2. the buckets' exclusive scan places them back to back;
//   3. scatter: the products are formed again and written to their
//      buckets as one 16-byte record each (key, residue; 32 bytes with the
//      two words of an int128 product), so a scattered product is one store;
//   4. one CTA per bucket at a time loads it into shared memory, sorts it
//      (block_sort_interval), sums equal keys and writes the non-zero terms
//      in ascending order to the bucket's part of the result arrays;
//   5. buckets with more products than shared memory holds are rare (a
//      bucket is sized for about 1024 products): each is sorted by a
//      device-wide radix sort of its keys' offsets and reduced by one CTA;
//   6. compaction concatenates the buckets in ascending order (K-e).
#include "pm_blocksort.cuh"
#include "pm_bucket.cuh"
#include "pm_partition.cuh"

namespace pm {

constexpr int GEN_T = 256;              // threads of the count and scatter kernels
constexpr int BK_T = 512;               // threads of the bucket kernel
constexpr u32 BK_CHUNK = 4096;          // products sorted per bucket in shared memory
constexpr int BK_IPT = BK_CHUNK / BK_T;
constexpr int BR_T = 1024;              // threads of the large-bucket reduction

// words of a bucketed product's record: key + residue, or key + int128 + pad
template <int WORDS>
__host__ __device__ constexpr u32 rec_words() { return WORDS == 1 ? 2u : 4u; }

struct BucketArgs {
    const u64 *A, *Ac, *B, *Bc;  // canonical f (rows) and g (columns): keys, coefficients
    u32 na, nb;
    u64 lo, end;                 // output keys [lo, end)
    const u64 *S;                // bucket b holds keys [S[b], S[b+1]); S[0] = lo, S[nbk] = end
    const u32 *T;                // T[t]: the bucket of key lo + t 2^tshift (t <= ncell)
    u32 tshift, ncell;
    u64 nbk;
    u64 *cnt;                    // products per bucket (count pass)
    u64 *fill;                   // fill counters (scatter pass)
    const u64 *boff;             // exclusive scan of cnt
    u64 *irec;                   // bucketed products: records of RW words {key, coefficient words}
    u64 *okey, *ocoef;           // results: bucket b's terms from boff[b] on, `words` words each
    u32 words;                   // 1 (mod p) or 2 (int64 products as int128)
    u64 *ucount;                 // result terms per bucket
    u32 *big;                    // [0]: buckets above the chunk; [1..]: their indexes
};

// the columns of row i whose products lie in [lo, end)
__device__ __forceinline__ void row_columns(const BucketArgs &a, u64 alpha, u32 &jl, u32 &jh)
{
    jl = a.lo > alpha ? lower_bound_u64(a.B, a.nb, a.lo - alpha) : 0u;
    jh = a.end > alpha ? lower_bound_u64(a.B, a.nb, a.end - alpha) : 0u;
}

// the bucket of a key in [lo, end): the table's cell gives the first and
// last candidate, a binary search over the boundaries between them the one
__device__ __forceinline__ u64 bucket_of(const BucketArgs &a, u64 key)
{
    const u64 t = (key - a.lo) >> a.tshift;
    u32 k = __ldg(a.T + t), hi = __ldg(a.T + t + 1);  // key's bucket is in [k, hi]
    while (k < hi) {
        const u32 mid = (k + hi + 1) >> 1;
        if (__ldg(a.S + mid) <= key) k = mid;
        else hi = mid - 1;
    }
    return k;
}

// lanes j0 + lane (valid ones a prefix) with ascending keys: the run of
// lanes sharing this lane's bucket -- its first lane and its length
__device__ __forceinline__ void bucket_run(bool valid, u64 b, u32 lane, u32 &head_lane, u32 &run_len, bool &head)
{
    const u32 vmask = __ballot_sync(0xffffffffu, valid);
    const u64 prev = __shfl_up_sync(0xffffffffu, b, 1);
    head = valid && (lane == 0 || prev != b);
    const u32 heads = __ballot_sync(0xffffffffu, head);
    const u32 upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    head_lane = 31u - (u32)__clz(heads & upto);
    const u32 after = lane == 31 ? 0u : (heads & (0xfffffffeu << lane));
    const u32 stop = after ? (u32)(__ffs(after) - 1) : (32u - (u32)__clz(vmask));
    run_len = stop - lane;
}

__global__ void __launch_bounds__(GEN_T) k_bucket_count(BucketArgs a)
{
    const u32 lane = threadIdx.x & 31;
    const u32 warps = gridDim.x * (GEN_T / 32);
    for (u32 i = (blockIdx.x * GEN_T + threadIdx.x) >> 5; i < a.na; i += warps) {
        const u64 alpha = __ldg(a.A + i);
        u32 jl, jh;
        row_columns(a, alpha, jl, jh);
        for (u32 j0 = jl; j0 < jh; j0 += 32) {
            const u32 j = j0 + lane;
            const bool valid = j < jh;
            const u64 b = valid ? bucket_of(a, alpha + __ldg(a.B + j)) : ~0ull;
            u32 hl, len;
            bool head;
            bucket_run(valid, b, lane, hl, len, head);
            if (head) atomicAdd(a.cnt + b, (u64)len);
        }
    }
}

template <int WORDS>
__global__ void __launch_bounds__(GEN_T) k_bucket_scatter(BucketArgs a)
{
    const u32 lane = threadIdx.x & 31;
    const u32 warps = gridDim.x * (GEN_T / 32);
    for (u32 i = (blockIdx.x * GEN_T + threadIdx.x) >> 5; i < a.na; i += warps) {
        const u64 alpha = __ldg(a.A + i), ca = __ldg(a.Ac + i);
        u32 jl, jh;
        row_columns(a, alpha, jl, jh);
        for (u32 j0 = jl; j0 < jh; j0 += 32) {
            const u32 j = j0 + lane;
            const bool valid = j < jh;
            const u64 key = valid ? alpha + __ldg(a.B + j) : 0;
            const u64 b = valid ? bucket_of(a, key) : ~0ull;
            u32 hl, len;
            bool head;
            bucket_run(valid, b, lane, hl, len, head);
            u64 at = 0;
            if (head) at = __ldg(a.boff + b) + atomicAdd(a.fill + b, (u64)len);
            at = __shfl_sync(0xffffffffu, at, hl);
            if (valid) {
                const u64 pos = at + (lane - hl);
                const u64 cb = __ldg(a.Bc + j);
                ulonglong2 *r = (ulonglong2 *)(a.irec + rec_words<WORDS>() * pos);
                if (WORDS == 1) {
                    r[0] = make_ulonglong2(key, m61_reduce(m61_mul_lazy(ca, cb)));
                } else {
                    u64 plo, phi;
                    mul_i64_wide((i64)ca, (i64)cb, plo, phi);
                    r[0] = make_ulonglong2(key, plo);
                    r[1] = make_ulonglong2(phi, 0ull);
                }
            }
        }
    }
}

// one bucket at a time per CTA: sort in shared memory, sum equal keys, write
// the bucket's terms in ascending order over its own items
template <int WORDS>
__global__ void __launch_bounds__(BK_T) k_bucket_sort(BucketArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 ws[32];
    u64 *kA = (u64 *)smem, *kB = kA + BK_CHUNK;
    u64 *cv = kB + BK_CHUNK;                                  // WORDS * BK_CHUNK words
    uint16_t *iA = (uint16_t *)(cv + WORDS * BK_CHUNK), *iB = iA + BK_CHUNK;
    u32 *hist = (u32 *)(iB + BK_CHUNK);                       // BUCKETS words
    const u32 tid = threadIdx.x;
    for (u64 b = blockIdx.x; b < a.nbk; b += gridDim.x) {
        const u64 n = a.cnt[b], base = a.boff[b];
        if (n > BK_CHUNK) {
            if (tid == 0) {
                const u32 k = atomicAdd(a.big, 1u);
                a.big[1 + k] = (u32)b;
                a.ucount[b] = 0;
            }
            continue;
        }
        const u64 blo = a.S[b], bspan = a.S[b + 1] - blo;
        u64 *kA_ = kA, *kB_ = kB;
        uint16_t *iA_ = iA, *iB_ = iB;
        for (u32 q = tid; q < n; q += BK_T) {
            const ulonglong2 *r = (const ulonglong2 *)(a.irec + rec_words<WORDS>() * (base + q));
            const ulonglong2 r0 = r[0];
            kA_[q] = r0.x - blo;
            iA_[q] = (uint16_t)q;
            cv[q] = r0.y;
            if (WORDS == 2) cv[BK_CHUNK + q] = r[1].x;
        }
        __syncthreads();
        block_sort_interval<BK_T, BK_IPT>(kA_, iA_, kB_, iB_, (u32)n, 0, bspan - 1, hist, ws);
        u64 run = 0;
        for (u32 c0 = 0; c0 < n; c0 += BK_T) {
            const u32 i = c0 + tid;
            u64 v0 = 0, v1 = 0;
            bool nz = false;
            if (i < n && (i == 0 || kA_[i] != kA_[i - 1])) {
                const u64 key = kA_[i];
                for (u32 jj = i; jj < n && kA_[jj] == key; jj++) {
                    const u32 src = iA_[jj];
                    if (WORDS == 1) v0 = m61_add(v0, cv[src]);
                    else add128(v0, v1, cv[src], cv[BK_CHUNK + src]);
                }
                nz = (v0 | v1) != 0;
            }
            u64 cnt;
            const u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, ws);
            if (nz) {
                const u64 d = base + run + pos;
                a.okey[d] = blo + kA_[i];
                a.ocoef[WORDS * d] = v0;
                if (WORDS == 2) a.ocoef[2 * d + 1] = v1;
            }
            run += cnt;
        }
        if (tid == 0) a.ucount[b] = run;
        __syncthreads();
    }
}

// a large bucket after its keys' offsets were sorted with the original
// positions as payload: sum equal keys (coefficients gathered from the
// records through the positions) into out (key, `words` words), one CTA;
// *count = terms written
template <int WORDS>
__global__ void __launch_bounds__(BR_T) k_bucket_big_reduce(const u64 *__restrict__ key, const u64 *__restrict__ idx,
                                                            const u64 *__restrict__ irec, u64 n, u64 blo,
                                                            u64 *__restrict__ okey, u64 *__restrict__ ocoef,
                                                            u64 *__restrict__ count)
{
    constexpr u32 RW = rec_words<WORDS>();
    __shared__ u64 ws[32];
    const u32 tid = threadIdx.x;
    u64 run = 0;
    for (u64 c0 = 0; c0 < n; c0 += BR_T) {
        const u64 i = c0 + tid;
        u64 v0 = 0, v1 = 0;
        bool nz = false;
        if (i < n && (i == 0 || key[i] != key[i - 1])) {
            const u64 k = key[i];
            for (u64 jj = i; jj < n && key[jj] == k; jj++) {
                const u64 s = idx[jj];
                if (WORDS == 1) v0 = m61_add(v0, irec[RW * s + 1]);
                else add128(v0, v1, irec[RW * s + 1], irec[RW * s + 2]);
            }
            nz = (v0 | v1) != 0;
        }
        u64 cnt;
        const u64 pos = block_exclusive_scan(nz ? 1 : 0, cnt, ws);
        if (nz) {
            okey[run + pos] = blo + key[i];
            ocoef[WORDS * (run + pos)] = v0;
            if (WORDS == 2) ocoef[WORDS * (run + pos) + 1] = v1;
        }
        run += cnt;
    }
    if (tid == 0) *count = run;
}

// a large bucket's keys as offsets from its first key, positions as the
// payload of the sort
__global__ void k_bucket_offsets(const u64 *__restrict__ irec, u32 rw, u64 *__restrict__ key, u64 *__restrict__ idx,
                                 u64 n, u64 blo)
{
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        key[i] = irec[rw * i] - blo;
        idx[i] = i;
    }
}

// bucket boundaries: every eighth of the sorted grid points (S[0] = lo,
// S[nbk] = end)
__global__ void k_bucket_bounds(const u64 *__restrict__ grid, u64 ngrid, u32 every, u64 nbk, u64 lo, u64 end,
                                u64 *__restrict__ S)
{
    const u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nbk) return;
    S[k] = k == 0 ? lo : (k == nbk ? end : grid[k * every]);
}

// T[t] = the bucket of key lo + t 2^tshift, for t = 0..ncell (clamped to
// the last bucket)
__global__ void k_bucket_table(const u64 *__restrict__ S, u64 nbk, u64 lo, u32 tshift, u32 ncell,
                               u32 *__restrict__ T)
{
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ncell) return;
    const u64 x = lo + ((u64)t << tshift);
    // last k in [0, nbk) with S[k] <= x
    u64 k = 0, len = nbk;
    while (len > 0) {
        const u64 half = len >> 1;
        if (S[k + half] <= x) {
            k += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    T[t] = (u32)(k ? k - 1 : 0);
}

template <class K>
static void set_smem_bk(K kernel, size_t bytes)
{
    PM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static size_t bucket_sort_smem(u32 words)
{
    return (size_t)BK_CHUNK * (8 + 8 + 8 * words + 2 + 2) + (size_t)BUCKETS * 4;
}

BucketSlices bucket_product(Ctx &c, Scratch &S, const BucketInputs &in, int kind, u64 lo, u64 end, u64 products)
{
    BucketSlices out;
    const u32 words = kind == PM_COEF_M61 ? 1u : 2u;
    // boundaries from the Sec. 5 grid: about eight sorted grid points per
    // bucket of about 1024 term products
    const u32 every = 8;
    const u64 want = products / 1024 + 1;
    u32 l = 1;
    while ((u64)(l + 1) * (l + 1) < every * want && l < 4096) l++;
    u32 ngrid = 0;
    const u64 *grid = grid_splitters(c, S, in.A, in.na, in.B, in.nb, l, in.A_last + in.B_last + 1, &ngrid, lo, end);
    // grid holds lo first and end last (clamped), ngrid >= 2
    const u64 nbk = ngrid > every ? (ngrid - 1) / every : 1;
    u64 *bounds = S.get<u64>(nbk + 1);
    k_bucket_bounds<<<(unsigned)((nbk + 256) / 256), 256, 0, c.s>>>(grid, ngrid, every, nbk, lo, end, bounds);
    PM_LAUNCHED(c);
    // lookup table over the top bits of key - lo: about four cells per bucket
    const u64 span = end - lo;
    int tb = 1;
    while (tb < 22 && (1ull << tb) < 4 * nbk) tb++;
    const int span_bits = bit_length(span - 1);
    const u32 tshift = span_bits > tb ? (u32)(span_bits - tb) : 0u;
    const u32 ncell = (u32)((span - 1) >> tshift) + 1;
    u32 *table = S.get<u32>((size_t)ncell + 1);
    k_bucket_table<<<(ncell + 256) / 256, 256, 0, c.s>>>(bounds, nbk, lo, tshift, ncell, table);
    PM_LAUNCHED(c);

    BucketArgs a;
    memset(&a, 0, sizeof(a));
    a.A = in.A;
    a.Ac = in.Ac;
    a.B = in.B;
    a.Bc = in.Bc;
    a.na = in.na;
    a.nb = in.nb;
    a.lo = lo;
    a.end = end;
    a.S = bounds;
    a.T = table;
    a.tshift = tshift;
    a.ncell = ncell;
    a.nbk = nbk;
    a.words = words;
    a.cnt = S.get<u64>(nbk);
    a.fill = S.get<u64>(nbk);
    u64 *boff = S.get<u64>(nbk + 1);
    a.boff = boff;
    a.ucount = S.get<u64>(nbk + 1);
    a.big = S.get<u32>(nbk + 1);
    PM_CUDA(cudaMemsetAsync(a.cnt, 0, nbk * 8, c.s));
    PM_CUDA(cudaMemsetAsync(a.fill, 0, nbk * 8, c.s));
    PM_CUDA(cudaMemsetAsync(a.big, 0, 4, c.s));
    const unsigned gen_grid = (unsigned)c.sm_count * 8;
    k_bucket_count<<<gen_grid, GEN_T, 0, c.s>>>(a);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, a.cnt, boff, nbk);
    u64 total = 0;
    PM_CUDA(cudaMemcpyAsync(&total, boff + nbk, 8, cudaMemcpyDeviceToHost, c.s));
    c.sync();
    const u32 rw = words == 1 ? rec_words<1>() : rec_words<2>();
    a.irec = S.get<u64>((total + 1) * rw);
    a.okey = S.get<u64>(total + 1);
    a.ocoef = S.get<u64>((total + 1) * words);
    if (words == 1) k_bucket_scatter<1><<<gen_grid, GEN_T, 0, c.s>>>(a);
    else k_bucket_scatter<2><<<gen_grid, GEN_T, 0, c.s>>>(a);
    PM_LAUNCHED(c);
    const size_t smem = bucket_sort_smem(words);
    const unsigned sort_grid = (unsigned)(nbk < (u64)c.sm_count ? nbk : (u64)c.sm_count);
    if (words == 1) {
        set_smem_bk(k_bucket_sort<1>, smem);
        k_bucket_sort<1><<<sort_grid, BK_T, smem, c.s>>>(a);
    } else {
        set_smem_bk(k_bucket_sort<2>, smem);
        k_bucket_sort<2><<<sort_grid, BK_T, smem, c.s>>>(a);
    }
    PM_LAUNCHED(c);
    // the buckets above the chunk: a device-wide sort each, then a reduction
    u32 nbig = 0;
    PM_CUDA(cudaMemcpyAsync(&nbig, a.big, 4, cudaMemcpyDeviceToHost, c.s));
    c.sync();
    out.big = nbig;
    if (nbig) {
        std::vector<u32> list(nbig);
        PM_CUDA(cudaMemcpyAsync(list.data(), a.big + 1, (size_t)nbig * 4, cudaMemcpyDeviceToHost, c.s));
        std::vector<u64> hcnt(nbk), hoff(nbk), hS(nbk + 1);
        PM_CUDA(cudaMemcpyAsync(hcnt.data(), a.cnt, nbk * 8, cudaMemcpyDeviceToHost, c.s));
        PM_CUDA(cudaMemcpyAsync(hoff.data(), boff, nbk * 8, cudaMemcpyDeviceToHost, c.s));
        PM_CUDA(cudaMemcpyAsync(hS.data(), bounds, (nbk + 1) * 8, cudaMemcpyDeviceToHost, c.s));
        c.sync();
        u64 nmax = 0;
        for (u32 b : list) nmax = hcnt[b] > nmax ? hcnt[b] : nmax;
        u64 *idx = S.get<u64>(nmax), *tkey = S.get<u64>(nmax);
        for (u32 b : list) {
            const u64 n = hcnt[b], base = hoff[b], blo = hS[b];
            k_bucket_offsets<<<(unsigned)((n + 255) / 256), 256, 0, c.s>>>(a.irec + rw * base, rw, tkey, idx, n, blo);
            PM_LAUNCHED(c);
            // the offsets lie in [0, S[b+1] - S[b])
            radix_sort_pairs(c, S, tkey, idx, nullptr, n, bit_length(hS[b + 1] - blo - 1));
            if (words == 1)
                k_bucket_big_reduce<1><<<1, BR_T, 0, c.s>>>(tkey, idx, a.irec + rw * base, n, blo, a.okey + base,
                                                            a.ocoef + base, a.ucount + b);
            else
                k_bucket_big_reduce<2><<<1, BR_T, 0, c.s>>>(tkey, idx, a.irec + rw * base, n, blo, a.okey + base,
                                                            a.ocoef + 2 * base, a.ucount + b);
            PM_LAUNCHED(c);
        }
    }
    out.n = nbk;
    out.key = a.okey;
    out.coef = a.ocoef;
    out.base = boff;
    out.ucount = a.ucount;
    out.words = words;
    return out;
}

}  // namespace pm
