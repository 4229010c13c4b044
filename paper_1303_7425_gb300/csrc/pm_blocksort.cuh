// Block-wide sorts of (key, index) pairs in shared memory: a stable LSD
// radix sort, and a bucket sort for keys drawn from a known interval.
#pragma once

#include "pm_common.cuh"

namespace pm {

// Sorts n <= THREADS * IPT pairs (kA[i], iA[i]) by the bits [0, nbits) of
// the key, 8 bits per pass.  Items are visited in index order (warp w owns
// a contiguous slice of 32 * ipt items, step s its s-th 32), so equal keys
// keep their order.  hist: THREADS / 32 * 256 words of shared memory, ws: 32
// words for block_exclusive_scan.  On return kA/iA point at the sorted
// buffers (the two buffers swap once per pass).  All threads must call.
template <int THREADS, int IPT, class I>
__device__ void block_sort_pairs(u64 *&kA, I *&iA, u64 *&kB, I *&iB, u32 n, int nbits, u32 *hist, u64 *ws)
{
    constexpr int W = THREADS / 32;
    const u32 tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const u32 ipt = (n + THREADS - 1) / THREADS;  // <= IPT
    for (int shift = 0; shift < nbits; shift += 8) {
        for (u32 x = tid; x < W * 256; x += THREADS) hist[x] = 0;
        __syncthreads();
        u32 rank[IPT], dig[IPT];
#pragma unroll
        for (int s = 0; s < IPT; s++) {
            if ((u32)s < ipt) {
                const u32 i = w * 32 * ipt + s * 32 + lane;
                const bool valid = i < n;
                const u32 d = valid ? (u32)((kA[i] >> shift) & 255u) : 256u;
                const u32 peers = __match_any_sync(0xffffffffu, d);
                const u32 lt = __popc(peers & ((1u << lane) - 1u));
                const u32 base = valid ? hist[w * 256 + d] : 0u;
                __syncwarp();
                if (valid && lt == 0) hist[w * 256 + d] = base + __popc(peers);
                __syncwarp();
                rank[s] = base + lt;
                dig[s] = d;
            }
        }
        __syncthreads();
        u64 dsum = 0;
        if (tid < 256) {
            u32 run = 0;
            for (int ww = 0; ww < W; ww++) {
                const u32 c = hist[ww * 256 + tid];
                hist[ww * 256 + tid] = run;
                run += c;
            }
            dsum = run;
        }
        u64 tot;
        const u64 dbase = block_exclusive_scan(dsum, tot, ws);
        if (tid < 256)
            for (int ww = 0; ww < W; ww++) hist[ww * 256 + tid] += (u32)dbase;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < IPT; s++) {
            if ((u32)s < ipt) {
                const u32 i = w * 32 * ipt + s * 32 + lane;
                if (i < n) {
                    const u32 pos = hist[w * 256 + dig[s]] + rank[s];
                    kB[pos] = kA[i];
                    iB[pos] = iA[i];
                }
            }
        }
        __syncthreads();
        u64 *tk = kA;
        kA = kB;
        kB = tk;
        I *ti = iA;
        iA = iB;
        iB = ti;
    }
}

// number of low bits in which the keys [k0, k0 + n) can differ
__device__ __forceinline__ int varying_bits(u64 lo, u64 hi_inclusive)
{
    u64 x = lo ^ hi_inclusive;
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

constexpr u32 BUCKETS = 4096;     // bucket-sort buckets (hist words it needs)
constexpr u32 BUCKET_RANK_MAX = 32;  // larger buckets: fall back to the radix sort

// Sorts n <= THREADS * IPT pairs whose keys lie in [lo, lo + span].  The
// pairs are distributed over 4096 buckets on the top 12 significant bits of
// key - lo; each pair then finds its place inside its bucket by counting
// the bucket's smaller keys (ties by position), so every pair moves twice
// and no thread works on more than one bucket's worth of compares per pair.
// When span < 4096 a bucket holds one key value and the scatter alone
// sorts.  For sparse products (keys spread over 50 and more bits) this
// replaces the 7 or 8 passes of an 8-bit radix sort.  Equal keys come out
// adjacent but in no particular order, so callers must only combine them
// with an exact (order-free) sum.  When a bucket holds more than
// BUCKET_RANK_MAX pairs (keys clustered inside the interval) the radix sort
// runs instead.  hist: at least max(4096, THREADS / 32 * 256) words; ws: 32
// words.  All threads must call.
template <int THREADS, int IPT, class I>
__device__ void block_sort_interval(u64 *&kA, I *&iA, u64 *&kB, I *&iB, u32 n, u64 lo, u64 span, u32 *hist,
                                    u64 *ws)
{
    static_assert(BUCKETS % THREADS == 0, "buckets per thread");
    constexpr u32 PER = BUCKETS / THREADS;
    __shared__ u32 s_bmax;
    const u32 tid = threadIdx.x, lane = tid & 31;
    int nb = 0;
    for (u64 x = span; x; x >>= 1) nb++;
    const int shift = nb > 12 ? nb - 12 : 0;
    for (u32 x = tid; x < BUCKETS; x += THREADS) hist[x] = 0;
    if (tid == 0) s_bmax = 0;
    __syncthreads();
    const u32 nround = (n + 31u) & ~31u;
    if (shift > 0) {
        // spread keys: few collisions, one atomic per pair
        for (u32 q = tid; q < n; q += THREADS) atomicAdd(&hist[(u32)min((kA[q] - lo) >> shift, (u64)BUCKETS - 1)], 1u);
    } else {
        // one key value per bucket, often repeated: one atomic per distinct
        // bucket of a warp
        for (u32 i = tid & ~31u; i < nround; i += THREADS) {
            const u32 q = i + lane;
            const bool valid = q < n;
            const u32 b = valid ? (u32)min(kA[q] - lo, (u64)BUCKETS - 1) : BUCKETS;
            const u32 peers = __match_any_sync(0xffffffffu, b);
            if (valid && lane == (u32)(__ffs(peers) - 1)) atomicAdd(&hist[b], (u32)__popc(peers));
        }
    }
    __syncthreads();
    // exclusive offsets (thread t owns buckets [t PER, t PER + PER)) and the
    // largest bucket
    u32 c[PER];
    u32 sum = 0, mx = 0;
#pragma unroll
    for (u32 q = 0; q < PER; q++) {
        c[q] = hist[tid * PER + q];
        sum += c[q];
        mx = c[q] > mx ? c[q] : mx;
    }
    if (mx > BUCKET_RANK_MAX) atomicMax(&s_bmax, mx);
    u64 tot;
    u32 run = (u32)block_exclusive_scan(sum, tot, ws);
#pragma unroll
    for (u32 q = 0; q < PER; q++) {
        hist[tid * PER + q] = run;
        run += c[q];
    }
    __syncthreads();
    if (shift > 0 && s_bmax > BUCKET_RANK_MAX) {
        block_sort_pairs<THREADS, IPT>(kA, iA, kB, iB, n, varying_bits(lo, lo + span), hist, ws);
        return;
    }
    // scatter; afterwards hist[b] is the end of bucket b
    if (shift > 0) {
        for (u32 q = tid; q < n; q += THREADS) {
            const u64 key = kA[q];
            const u32 b = (u32)min((key - lo) >> shift, (u64)BUCKETS - 1);
            const u32 pos = atomicAdd(&hist[b], 1u);
            kB[pos] = key;
            iB[pos] = iA[q];
        }
    } else {
        for (u32 i = tid & ~31u; i < nround; i += THREADS) {
            const u32 q = i + lane;
            const bool valid = q < n;
            const u64 key = valid ? kA[q] : 0;
            const u32 b = valid ? (u32)min(key - lo, (u64)BUCKETS - 1) : BUCKETS;
            const u32 peers = __match_any_sync(0xffffffffu, b);
            const u32 leader = (u32)(__ffs(peers) - 1);
            u32 base = 0;
            if (valid && lane == leader) base = atomicAdd(&hist[b], (u32)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (valid) {
                const u32 pos = base + (u32)__popc(peers & ((1u << lane) - 1u));
                kB[pos] = key;
                iB[pos] = iA[q];
            }
        }
    }
    __syncthreads();
    if (shift == 0) {
        u64 *tk = kA;
        kA = kB;
        kB = tk;
        I *ti = iA;
        iA = iB;
        iB = ti;
        return;
    }
    // rank inside the bucket, written back to the A buffers
    for (u32 x = tid; x < n; x += THREADS) {
        const u64 key = kB[x];
        const u32 b = (u32)min((key - lo) >> shift, (u64)BUCKETS - 1);
        const u32 beg = b ? hist[b - 1] : 0u, end = hist[b];
        u32 rank = 0;
        for (u32 y = beg; y < end; y++) {
            const u64 o = kB[y];
            rank += (o < key || (o == key && y < x)) ? 1u : 0u;
        }
        kA[beg + rank] = key;
        iA[beg + rank] = iB[x];
    }
    __syncthreads();
}

}  // namespace pm
