// Register-only rate probe of the per-term-product arithmetic
// (include/polymul_probe.h).
#include "pm_common.cuh"
#include "polymul_probe.h"

namespace pm {

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

}  // namespace pm

extern "C" int pm_probe_mac(uint32_t blocks, uint32_t threads, uint64_t iters, uint64_t seed, uint64_t *sink,
                            void *stream)
{
    if (!blocks || !threads || threads > 1024 || !sink) return PM_EINVAL;
    pm::k_probe_mac<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, seed, (pm::u64 *)sink);
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}
