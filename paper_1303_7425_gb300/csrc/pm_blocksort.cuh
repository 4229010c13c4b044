// Block-wide stable LSD radix sort of (key, index) pairs in shared memory.
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

}  // namespace pm
