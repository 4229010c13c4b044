/* polymul_probe.h -- measurement probes for the roofline of the product's
 * accumulate kernels (libpolymul_probe.so, a library of its own; the
 * product's C-ABI in polymul.h does not include them).
 *
 * The paper has no counterpart.  These are register-only microkernels:
 *   pm_probe_mac     the per-term-product arithmetic in one loop (one 64-bit
 *                    key add, the 61 x 61 -> 122-bit product, the Mersenne
 *                    fold, one modular add) plus a 64-bit add and a mask per
 *                    product that advance the operand;
 *   pm_probe_oprate  the throughput of one integer instruction class at a
 *                    time (32 x 32 -> 64 multiply-add, 32-bit multiply-add,
 *                    three-input add, three-input logic op, funnel shift,
 *                    high half of a 32 x 32 multiply), from which the
 *                    benchmark derives the integer-op bound per term product
 *                    (4 wide multiplies + 14 simple ops).
 */
#ifndef POLYMUL_PROBE_H
#define POLYMUL_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* instruction classes of pm_probe_oprate */
#define PM_OP_IMAD_WIDE 0  /* mad.wide.u32: 32 x 32 -> 64 multiply-add          */
#define PM_OP_IMAD      1  /* mad.lo.u32: 32-bit multiply-add                    */
#define PM_OP_IADD3     2  /* three-input 32-bit add                             */
#define PM_OP_LOP3      3  /* three-input 32-bit logic op                        */
#define PM_OP_SHF       4  /* 32-bit funnel shift                                */
#define PM_OP_IMAD_HI   6  /* mad.hi.u32: high half of a 32 x 32 multiply, added */

/* Launch blocks x threads threads; each performs `iters` iterations of 4
 * independent multiply-accumulate chains (4 * iters term products) and
 * writes one checksum word to sink[block * threads + thread] (device
 * memory of blocks * threads uint64).  Returns 0 or -1 (bad arguments) /
 * -7 (launch failed).  Time it with CUDA events on `stream`. */
int pm_probe_mac(uint32_t blocks, uint32_t threads, uint64_t iters, uint64_t seed, uint64_t *sink, void *stream);

/* Launch blocks x threads threads of the probe for instruction class `op`;
 * each thread runs `iters` steps of pm_probe_ops_per_step(op) instructions
 * of that class, on independent register chains whose operands change every
 * step, and writes one checksum word to sink[block * threads + thread]
 * (device, blocks * threads uint64).  clk (device, 2 uint64, or NULL)
 * receives the first block's SM clock cycles and global-timer nanoseconds
 * from its entry to its exit, i.e. the SM clock the probe ran at.  Returns
 * 0, -1 (bad arguments or op) or -7 (launch failed). */
int pm_probe_oprate(int op, uint32_t blocks, uint32_t threads, uint64_t iters, uint32_t seed, uint64_t *sink,
                    uint64_t *clk, void *stream);

/* Instructions one thread issues per step of pm_probe_oprate(op); 0 for an
 * unknown op. */
uint32_t pm_probe_ops_per_step(int op);

#ifdef __cplusplus
}
#endif
#endif
