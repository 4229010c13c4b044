/* polymul_probe.h -- measurement helper for the library's roofline.
 *
 * The paper has no counterpart: this is a register-only microkernel that
 * measures how many exact term products per second the GPU's integer
 * pipelines can do when a term product costs only its algorithmic
 * arithmetic (one 64-bit key add, the 61 x 61 -> 122-bit product, the
 * Mersenne fold, one modular add).  The benchmark divides the range
 * kernel's achieved rate by this figure.
 */
#ifndef POLYMUL_PROBE_H
#define POLYMUL_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Launch blocks x threads threads; each performs `iters` iterations of 4
 * independent multiply-accumulate chains (4 * iters term products) and
 * writes one checksum word to sink[block * threads + thread] (device
 * memory of blocks * threads uint64).  Returns 0 or PM_EINVAL / PM_ECUDA.
 * Time it with CUDA events on `stream`. */
int pm_probe_mac(uint32_t blocks, uint32_t threads, uint64_t iters, uint64_t seed, uint64_t *sink, void *stream);

#ifdef __cplusplus
}
#endif
#endif
