// Device primitives used by the host driver: exclusive scan of uint64 arrays
// and a stable LSD radix sort of (uint64 key, uint64 payloads).  Both are
// plain multi-kernel formulations sized in multiples of the tile; they run on
// the operands (n_f + n_g terms) and on the splitter arrays, never on the
// n_f * n_g term products.
#include "pm_common.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// exclusive scan
// ---------------------------------------------------------------------------

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const u64 *__restrict__ in, size_t n,
                                                              u64 *__restrict__ sums)
{
    __shared__ u64 ws[32];
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_IPT;
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++)
        if (base + k < n) s += in[base + k];
    u64 total;
    block_exclusive_scan(s, total, ws);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = offset(block) + exclusive prefix; the block holding element n-1
// also writes out[n] = grand total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const u64 *__restrict__ in, size_t n,
                                                             u64 *__restrict__ out,
                                                             const u64 *__restrict__ tile_offsets)
{
    __shared__ u64 ws[32];
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_IPT;
    u64 v[SCAN_IPT];
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    u64 total;
    u64 run = block_exclusive_scan(s, total, ws) + (tile_offsets ? tile_offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    size_t tile_end = (size_t)(blockIdx.x + 1) * SCAN_TILE;
    if (threadIdx.x == 0 && tile_end >= n)
        out[n] = total + (tile_offsets ? tile_offsets[blockIdx.x] : 0);
}

void scan_exclusive_u64(Ctx &c, Scratch &S, const u64 *in, u64 *out, size_t n)
{
    if (n == 0) {
        PM_CUDA(cudaMemsetAsync(out, 0, sizeof(u64), c.s));
        return;
    }
    size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, c.s>>>(in, n, out, nullptr);
        PM_LAUNCHED(c);
        return;
    }
    u64 *sums = S.get<u64>(nb);
    u64 *sums_ex = S.get<u64>(nb + 1);
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, c.s>>>(in, n, sums);
    PM_LAUNCHED(c);
    scan_exclusive_u64(c, S, sums, sums_ex, nb);
    k_scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, c.s>>>(in, n, out, sums_ex);
    PM_LAUNCHED(c);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 16;
constexpr int RS_TILE = RS_THREADS * RS_IPT;  // 4096 items per block

// per-block digit counts, stored digit-major: hist[d * nb + b]
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const u64 *__restrict__ keys, size_t n, int shift,
                                                        u64 *__restrict__ hist, unsigned nb)
{
    __shared__ u32 cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        size_t i = base + k;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Items of a tile are visited in index order (warp w owns a contiguous
// 512-item slice, step s the s-th 32 items of it), so ranks are stable.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const u64 *__restrict__ kin, const u64 *__restrict__ ain,
                                                           const u64 *__restrict__ bin, u64 *__restrict__ kout,
                                                           u64 *__restrict__ aout, u64 *__restrict__ bout, size_t n,
                                                           int shift, const u64 *__restrict__ offs, unsigned nb)
{
    __shared__ u32 whist[RS_WARPS][257];
    __shared__ u64 goff[256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) whist[ww][tid] = 0;
    goff[tid] = offs[(size_t)tid * nb + blockIdx.x];
    __syncthreads();

    const size_t tile0 = (size_t)blockIdx.x * RS_TILE + (size_t)w * (32 * RS_IPT);
    u32 rank[RS_IPT];
    u32 dig[RS_IPT];
#pragma unroll
    for (int s = 0; s < RS_IPT; s++) {
        size_t i = tile0 + (size_t)s * 32 + lane;
        bool valid = i < n;
        u32 d = valid ? (u32)((kin[i] >> shift) & 255u) : 256u;
        u32 peers = __match_any_sync(0xffffffffu, d);
        u32 lt = __popc(peers & ((1u << lane) - 1u));
        u32 base = valid ? whist[w][d] : 0u;
        __syncwarp();
        if (valid && lt == 0) whist[w][d] = base + __popc(peers);
        __syncwarp();
        rank[s] = base + lt;
        dig[s] = d;
    }
    __syncthreads();
    {
        u32 run = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ww++) {
            u32 c = whist[ww][tid];
            whist[ww][tid] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < RS_IPT; s++) {
        size_t i = tile0 + (size_t)s * 32 + lane;
        if (i < n) {
            u32 d = dig[s];
            size_t pos = goff[d] + whist[w][d] + rank[s];
            kout[pos] = kin[i];
            if (ain) aout[pos] = ain[i];
            if (bin) bout[pos] = bin[i];
        }
    }
}

void radix_sort_pairs(Ctx &c, Scratch &S, u64 *keys, u64 *v0, u64 *v1, size_t n, int nbits)
{
    if (n <= 1 || nbits <= 0) return;
    unsigned nb = (unsigned)((n + RS_TILE - 1) / RS_TILE);
    u64 *k2 = S.get<u64>(n);
    u64 *a2 = v0 ? S.get<u64>(n) : nullptr;
    u64 *b2 = v1 ? S.get<u64>(n) : nullptr;
    u64 *hist = S.get<u64>((size_t)256 * nb);
    u64 *offs = S.get<u64>((size_t)256 * nb + 1);
    u64 *ki = keys, *ai = v0, *bi = v1, *ko = k2, *ao = a2, *bo = b2;
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += 8, passes++) {
        k_rs_hist<<<nb, RS_THREADS, 0, c.s>>>(ki, n, shift, hist, nb);
        PM_LAUNCHED(c);
        scan_exclusive_u64(c, S, hist, offs, (size_t)256 * nb);
        k_rs_scatter<<<nb, RS_THREADS, 0, c.s>>>(ki, ai, bi, ko, ao, bo, n, shift, offs, nb);
        PM_LAUNCHED(c);
        std::swap(ki, ko);
        std::swap(ai, ao);
        std::swap(bi, bo);
    }
    if (passes & 1) {
        PM_CUDA(cudaMemcpyAsync(keys, ki, n * sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
        if (v0) PM_CUDA(cudaMemcpyAsync(v0, ai, n * sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
        if (v1) PM_CUDA(cudaMemcpyAsync(v1, bi, n * sizeof(u64), cudaMemcpyDeviceToDevice, c.s));
    }
}

}  // namespace pm
