// Shared device helpers of the polymul library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "polymul.h"

namespace pm {

typedef unsigned long long u64;
typedef long long i64;
typedef unsigned int u32;

constexpr u64 P61 = 0x1FFFFFFFFFFFFFFFull;  // 2^61 - 1

// status bits written by kernels, read by the host at the end of a step
constexpr u32 ST_EXP_OVERFLOW = 1u;
constexpr u32 ST_COEF_BOUND = 2u;
constexpr u32 ST_CAPACITY = 4u;
constexpr u32 ST_INTERNAL = 8u;

// ---------------------------------------------------------------------------
// arithmetic mod p = 2^61 - 1.  2^61 = 1 (mod p), so a 122-bit product
// hi * 2^64 + lo splits into (bits >= 61) + (bits < 61) with one add.
// ---------------------------------------------------------------------------

// a, b < 2^61: returns r < 2^62 with r = a*b (mod p)
__device__ __forceinline__ u64 m61_mul_lazy(u64 a, u64 b)
{
    u64 lo = a * b;
    u64 hi = __umul64hi(a, b);
    return (lo & P61) + ((hi << 3) | (lo >> 61));
}

// a b mod p from 31-bit splits, four 32 x 32 -> 64 multiplies.  With
// a = ah 2^31 + al and b = bh 2^31 + bl (al, bl < 2^31; ah, bh < 2^30),
//     a b = ah bh 2^62 + (ah bl + al bh) 2^31 + al bl,
// and 2^62 = 2, 2^61 = 1 (mod p); the middle sum m < 2^62 splits as
// m = mh 2^30 + ml (ml < 2^30), so m 2^31 = mh + ml 2^31 (mod p):
//     a b = al bl + 2 ah bh + mh + ml 2^31  (mod p), the sum < 2^64.
// as = al | ah << 32 (m61_split_row), bs = bl | (2 bh) << 32
// (m61_split_col): the doubled bh folds the 2 into one multiply.
__device__ __forceinline__ u64 m61_split_row(u64 a) { return (a & 0x7FFFFFFFull) | ((a >> 31) << 32); }
__device__ __forceinline__ u64 m61_split_col(u64 b) { return (b & 0x7FFFFFFFull) | ((b >> 31) << 33); }
__device__ __forceinline__ u64 m61_mul_split(u64 as, u64 bs)
{
    const u32 al = (u32)as, ah = (u32)(as >> 32), bl = (u32)bs, bh2 = (u32)(bs >> 32);
    const u64 t = (u64)al * bl + (u64)ah * bh2;
    const u64 m = (u64)ah * bl + (u64)al * (bh2 >> 1);
    return t + (m >> 30) + ((m & 0x3FFFFFFFull) << 31);
}

// a b mod p with three 32 x 32 -> 64 multiplies (Karatsuba's middle term):
// with a = al + ah 2^31, b = bl + bh 2^31 (al, bl < 2^31; ah, bh < 2^30),
//     ah bl + al bh = (al + ah)(bl + bh) - al bl - ah bh = m  (< 2^62),
// where (al + ah)(bl + bh) < 2^64 fits; as in m61_mul_split,
//     a b = al bl + 2 ah bh + mh + ml 2^31  (mod p),  m = mh 2^30 + ml,
// and the sum is below 2^63 + 2^62.  sa = al + ah and sb = bl + bh come
// precomputed with the halves.
__device__ __forceinline__ u64 m61_mul_k3(u32 al, u32 ah, u32 sa, u32 bl, u32 bh, u32 sb)
{
    const u64 p1 = (u64)al * bl, p2 = (u64)ah * bh, p3 = (u64)sa * sb;
    const u64 m = p3 - p1 - p2;
    return p1 + 2 * p2 + (m >> 30) + ((m & 0x3FFFFFFFull) << 31);
}

// any 64-bit x -> [0, p)
__device__ __forceinline__ u64 m61_reduce(u64 x)
{
    u64 r = (x & P61) + (x >> 61);  // <= p + 7
    return r >= P61 ? r - P61 : r;
}

// a, b in [0, p) -> a + b mod p
__device__ __forceinline__ u64 m61_add(u64 a, u64 b)
{
    u64 r = a + b;
    return r >= P61 ? r - P61 : r;
}

// 2^64 = 2^3 * 2^61 = 8 (mod p): adding into a wrapping 64-bit word stays
// exact mod p if every wrap is followed by an add of 8.
__device__ __forceinline__ void m61_atomic_accumulate(u64 *slot, u64 v)
{
    u64 old = atomicAdd(slot, v);
    u64 add = (old + v < old) ? 8ull : 0ull;
    while (add) {
        old = atomicAdd(slot, add);
        add = (old + add < old) ? 8ull : 0ull;
    }
}

// signed 64 x 64 -> 128 product as (lo, hi) words
__device__ __forceinline__ void mul_i64_wide(i64 a, i64 b, u64 &lo, u64 &hi)
{
    lo = (u64)a * (u64)b;
    hi = (u64)__mul64hi(a, b);
}

__device__ __forceinline__ void add128(u64 &lo, u64 &hi, u64 blo, u64 bhi)
{
    u64 l = lo + blo;
    hi = hi + bhi + (l < lo ? 1ull : 0ull);
    lo = l;
}

// (w0, w1, w2) += (x0, x1, x2), 192-bit two's complement words
__device__ __forceinline__ void add192w(u64 &w0, u64 &w1, u64 &w2, u64 x0, u64 x1, u64 x2)
{
    const u64 l = w0 + x0;
    const u64 c0 = l < w0 ? 1ull : 0ull;
    const u64 t = x1 + c0;                   // may wrap: then it carries one more
    const u64 c1a = t < x1 ? 1ull : 0ull;
    const u64 m = w1 + t;
    const u64 c1b = m < w1 ? 1ull : 0ull;
    w0 = l;
    w1 = m;
    w2 = w2 + x2 + c1a + c1b;
}

// (w0, w1, w2) += the int128 (blo, bhi) sign-extended to 192 bits
__device__ __forceinline__ void add192(u64 &w0, u64 &w1, u64 &w2, u64 blo, u64 bhi)
{
    add192w(w0, w1, w2, blo, bhi, (u64)((i64)bhi >> 63));
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan (all threads of the block must call it)
// ---------------------------------------------------------------------------

// one value per thread; returns the thread's exclusive prefix and sets
// `total` to the block's sum.  warp_sums: 32 words of shared memory.
__device__ __forceinline__ u64 block_exclusive_scan(u64 v, u64 &total, u64 *warp_sums)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u64 y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        u64 s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            u64 y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    u64 wbase = w > 0 ? warp_sums[w - 1] : 0;
    total = warp_sums[nw - 1];
    __syncthreads();
    return wbase + x - v;
}

// ---------------------------------------------------------------------------
// searches over sorted uint64 arrays
// ---------------------------------------------------------------------------

// first index i in [0, n) with a[i] >= x (n if none)
__device__ __forceinline__ u32 lower_bound_u64(const u64 *__restrict__ a, u32 n, u64 x)
{
    u32 lo = 0, len = n;
    while (len > 0) {
        u32 half = len >> 1;
        if (__ldg(a + lo + half) < x) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// ---------------------------------------------------------------------------
// exponent layout passed by value to kernels
// ---------------------------------------------------------------------------

struct Layout {
    u32 nv;
    u32 off[PM_MAX_VARS];     // bit offset of x_v's field (x_1 most significant)
    u32 width[PM_MAX_VARS];   // field width incl. guard bit
    u64 stride[PM_MAX_VARS];  // mixed-radix stride of x_v in the rank box
    u64 extent[PM_MAX_VARS];  // rank box extent of x_v
    // division by extent[v] < 2^32 as a multiply-high and two shifts
    // (set with the extents, see fastdiv_params)
    u32 dmag[PM_MAX_VARS];
    u32 dsh[PM_MAX_VARS];     // sh1 | sh2 << 8
};

// Division of a 32-bit n by an invariant 1 <= d < 2^32 with one multiply-
// high (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, sh1 = min(l, 1), sh2 = max(l - 1, 0),
// t = mulhi(m, n) and q = (t + ((n - t) >> sh1)) >> sh2 = floor(n / d).
inline void fastdiv_params(u64 d, u32 &m, u32 &sh)
{
    if (d == 0 || d > 0xFFFFFFFFull) {
        m = 0;
        sh = 0;
        return;
    }
    u32 l = 0;
    while ((1ull << l) < d) l++;
    const unsigned __int128 num = ((unsigned __int128)1 << 32) * (((unsigned __int128)1 << l) - d);
    m = (u32)(num / d + 1);
    const u32 sh1 = l < 1 ? l : 1, sh2 = l > 1 ? l - 1 : 0;
    sh = sh1 | (sh2 << 8);
}

__device__ __forceinline__ u32 fastdiv(u32 n, u32 m, u32 sh)
{
    const u32 t = __umulhi(m, n);
    return (t + ((n - t) >> (sh & 0xFF))) >> (sh >> 8);
}

__device__ __forceinline__ u32 key_field(const Layout &L, u64 key, u32 v)
{
    return (u32)((key >> L.off[v]) & ((1ull << L.width[v]) - 1ull));
}

__device__ __forceinline__ u64 key_to_rank(const Layout &L, u64 key)
{
    u64 r = 0;
    for (u32 v = 0; v < L.nv; v++) r += (u64)key_field(L, key, v) * L.stride[v];
    return r;
}

// rank -> packed key, for ranks inside the box
__device__ __forceinline__ u64 rank_to_key(const Layout &L, u64 rank)
{
    u64 key = 0;
    if (rank <= 0xFFFFFFFFull) {
        // extents are below 2^32 (fields of at most 32 bits, guard bit
        // included), so the fast division applies
        u32 r = (u32)rank;
        for (int v = (int)L.nv - 1; v >= 0; v--) {
            const u32 e = (u32)L.extent[v];
            const u32 q = fastdiv(r, L.dmag[v], L.dsh[v]);
            key |= (u64)(r - q * e) << L.off[v];
            r = q;
        }
    } else {
        for (int v = (int)L.nv - 1; v >= 0; v--) {
            u64 q = rank / L.extent[v];
            key |= (rank - q * L.extent[v]) << L.off[v];
            rank = q;
        }
    }
    return key;
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define PM_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::pm::Error(e_ == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA,       \
                              std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

#define PM_LAUNCHED(ctx)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess)                                                             \
            throw ::pm::Error(PM_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
        (ctx).launches++;                                                                  \
    } while (0)

// A caller-provided device workspace carved by a host-side bump pointer
// (pm_polymul_ws): blocks are 256-byte aligned and never freed; running
// past the end is PM_ENOMEM before any kernel touches the block.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    size_t used = 0;
};

// Where a call's scratch comes from: the stream-ordered pool (default),
// optionally adding every block's bytes to *tally (the workspace size
// query), or a caller's arena (no allocation at all).
struct ScratchMode {
    Arena *arena = nullptr;
    u64 *tally = nullptr;
};

inline size_t scratch_block_bytes(size_t bytes) { return bytes < 256 ? 256 : (bytes + 255) & ~(size_t)255; }

// Stream-ordered scratch: every block comes from cudaMallocAsync on the call's
// stream and goes back with cudaFreeAsync when the call ends -- or, in arena
// mode, from the caller's workspace.
struct Scratch {
    cudaStream_t s;
    ScratchMode mode;
    std::vector<void *> blocks;
    explicit Scratch(cudaStream_t st, ScratchMode m = ScratchMode()) : s(st), mode(m) {}
    ~Scratch()
    {
        for (void *p : blocks) cudaFreeAsync(p, s);
    }
    template <class T>
    T *get(size_t n)
    {
        const size_t bytes = scratch_block_bytes(n * sizeof(T));
        if (mode.arena) {
            Arena &a = *mode.arena;
            if (bytes > a.size - a.used) throw Error(PM_ENOMEM, "workspace too small");
            void *p = a.base + a.used;
            a.used += bytes;
            return (T *)p;
        }
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error(PM_ENOMEM, "cudaMallocAsync failed");
        }
        blocks.push_back(p);
        if (mode.tally) *mode.tally += bytes;
        return (T *)p;
    }
};

struct Ctx {
    cudaStream_t s;
    u32 launches = 0;
    u32 syncs = 0;
    int sm_count = 148;
    void sync()
    {
        PM_CUDA(cudaStreamSynchronize(s));
        syncs++;
    }
};

inline u32 ceil_div_u32(u64 a, u64 b) { return (u32)((a + b - 1) / b); }

inline int bit_length(u64 x)
{
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// device primitives (pm_prims.cu)
void scan_exclusive_u64(Ctx &c, Scratch &S, const u64 *in, u64 *out, size_t n);
void radix_sort_pairs(Ctx &c, Scratch &S, u64 *keys, u64 *v0, u64 *v1, size_t n, int nbits);

}  // namespace pm
