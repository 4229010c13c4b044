// Register-only rate probes for the roofline of the accumulate kernels
// (include/polymul_probe.h).  Built into libpolymul_probe.so, a measurement
// library of its own: the product's C-ABI (libpolymul.so) does not carry it.
#include "pm_common.cuh"
#include "polymul_probe.h"

namespace pm {

// Clock record of one thread of the first block: SM clock counter and the
// global nanosecond timer at entry and exit, so the host can turn the
// kernel's event time into SM cycles at the clock the SM actually ran.
__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct ClockRec {
    u64 *out;
    u64 c0, t0;
    __device__ __forceinline__ void start(u64 *o)
    {
        out = o;
        if (out && blockIdx.x == 0 && threadIdx.x == 0) {
            t0 = global_ns();
            c0 = clock64();
        }
    }
    __device__ __forceinline__ void stop()
    {
        if (out && blockIdx.x == 0 && threadIdx.x == 0) {
            const u64 c1 = clock64(), t1 = global_ns();
            out[0] = c1 - c0;
            out[1] = t1 - t0;
        }
    }
};

// ---------------------------------------------------------------------------
// The per-term-product arithmetic in one loop: key add, 61 x 61 -> 122-bit
// product, Mersenne fold, modular add; the operand b then advances by one
// 64-bit add and a mask (two simple ops per product beyond the algorithmic
// ones, which the op-rate probes below do not carry).
// ---------------------------------------------------------------------------
__global__ void k_probe_mac(u64 iters, u64 seed, u64 *__restrict__ sink)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 a[4], b[4], key[4], acc[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        a[c] = (seed * (t + 1) + 0x9E3779B97F4A7C15ull * c) & P61;
        b[c] = (seed ^ (t * 0xBF58476D1CE4E5B9ull + c)) & P61;
        key[c] = t + c;
        acc[c] = 0;
    }
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            key[c] += b[c];                                   // monomial product: one add
            u64 v = m61_mul_lazy(a[c], b[c]);                 // 122-bit product + fold
            acc[c] = m61_reduce(acc[c] + v);                  // modular accumulate
            b[c] = (b[c] + key[c]) & P61;                     // next operand
        }
    }
    sink[t] = acc[0] ^ acc[1] ^ acc[2] ^ acc[3] ^ key[0] ^ key[3];
}

// ---------------------------------------------------------------------------
// Op-rate probes: CH independent dependency chains per thread, one
// instruction of the measured class per chain step, operands that change
// every step (nothing can be hoisted out of the loop or folded).
// ---------------------------------------------------------------------------
constexpr int CH = 8;

// 32 x 32 -> 64 multiply-add: x_c <- hi(x_{c+1}) * b + x_c (the multiplicand
// comes from the next chain's high word, so no register of the product's
// pair is read and written by the same instruction)
__global__ void k_rate_imad_wide(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[CH];
    const u32 b = seed | 1u;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = (u64)(t * 2654435761u + c) << 1;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++)
            asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(x[c]) : "r"((u32)(x[(c + 1) % CH] >> 32)), "r"(b));
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

// 32-bit multiply-add: x <- x * b + c
__global__ void k_rate_imad(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 x[CH];
    const u32 b = seed | 1u, d = seed >> 7;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + c;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(b), "r"(d));
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

// three-input add: x_c <- x_c + x_{c+1} + d (the chains feed each other, so
// no sum can be re-associated away)
__global__ void k_rate_iadd3(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 x[CH];
    const u32 d = seed;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + c;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            u32 y = x[(c + 1) % CH];
            asm volatile("{ .reg .u32 q; add.u32 q, %0, %1; add.u32 %0, q, %2; }" : "+r"(x[c]) : "r"(y), "r"(d));
        }
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

// three-input logic op: x_c <- x_c ^ x_{c+1} ^ d
__global__ void k_rate_lop3(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 x[CH];
    const u32 d = seed;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + c;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            u32 y = x[(c + 1) % CH];
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(y), "r"(d));
        }
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

// funnel shift: x_c <- shf.l(x_c, x_{c+1}, d)
__global__ void k_rate_shf(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 x[CH];
    const u32 d = (seed & 15u) + 3u;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + c;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) {
            u32 y = x[(c + 1) % CH];
            asm volatile("shf.l.wrap.b32 %0, %1, %0, %2;" : "+r"(x[c]) : "r"(y), "r"(d));
        }
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

// high half of a 32 x 32 multiply: x <- mulhi(x, b) + x (the add keeps the
// chain from collapsing to zero)
__global__ void k_rate_imad_hi(u64 iters, u32 seed, u64 *__restrict__ sink, u64 *clk)
{
    ClockRec cr;
    cr.start(clk);
    const u32 t = blockIdx.x * blockDim.x + threadIdx.x;
    u32 x[CH];
    const u32 b = seed | 0x80000001u;
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = t * 2654435761u + c;
    for (u64 i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) asm volatile("mad.hi.u32 %0, %0, %1, %0;" : "+r"(x[c]) : "r"(b));
    }
    u32 s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s ^= x[c];
    sink[t] = s;
    cr.stop();
}

}  // namespace pm

extern "C" int pm_probe_mac(uint32_t blocks, uint32_t threads, uint64_t iters, uint64_t seed, uint64_t *sink,
                            void *stream)
{
    if (!blocks || !threads || threads > 1024 || !sink) return PM_EINVAL;
    pm::k_probe_mac<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, seed, (pm::u64 *)sink);
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

extern "C" int pm_probe_oprate(int op, uint32_t blocks, uint32_t threads, uint64_t iters, uint32_t seed,
                               uint64_t *sink, uint64_t *clk, void *stream)
{
    if (!blocks || !threads || threads > 1024 || !sink) return PM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    pm::u64 *k = (pm::u64 *)sink, *c = (pm::u64 *)clk;
    switch (op) {
    case PM_OP_IMAD_WIDE: pm::k_rate_imad_wide<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    case PM_OP_IMAD: pm::k_rate_imad<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    case PM_OP_IADD3: pm::k_rate_iadd3<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    case PM_OP_LOP3: pm::k_rate_lop3<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    case PM_OP_SHF: pm::k_rate_shf<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    case PM_OP_IMAD_HI: pm::k_rate_imad_hi<<<blocks, threads, 0, s>>>(iters, seed, k, c); break;
    default: return PM_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

extern "C" uint32_t pm_probe_ops_per_step(int op)
{
    switch (op) {
    case PM_OP_IMAD_WIDE:
    case PM_OP_IMAD:
    case PM_OP_IADD3:
    case PM_OP_LOP3:
    case PM_OP_SHF:
    case PM_OP_IMAD_HI: return pm::CH;
    default: return 0;
    }
}
