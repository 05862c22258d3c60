/*
 * bn_probe.h - measurement helper for the integer-multiply roofline.
 *
 * The multiplication kernels are bound by the integer multiply-add pipe, and
 * no peak for it is recorded for this GPU.  This entry point runs a
 * register-only kernel of independent multiply-add chains so a benchmark can
 * time it and derive the chip's 32-bit multiply-add rate per clock.  The
 * paper has no counterpart (its experiments time whole kernels only).
 */
#ifndef BN_GB300_PROBE_H
#define BN_GB300_PROBE_H

#include <stdint.h>

#include "bn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bn_probe_kind {
    BN_PROBE_MAD_LO = 0,      /* mad.lo.u32: 1 multiply-add per op */
    BN_PROBE_MAD_HI = 1,      /* mad.hi.u32 */
    BN_PROBE_MAD_WIDE = 2,    /* mad.wide.u32 (32x32 -> 64 plus a 64-bit addend) */
    BN_PROBE_MAC_CHAIN = 3    /* the schoolbook kernel's inner step: an 8-word mad.lo
                                 carry chain and an 8-word mad.hi carry chain */
} bn_probe_kind;

/* Enqueue the probe: `blocks` x `threads` threads each run `iters` iterations
 * of 8 independent multiply-adds of the given kind (for BN_PROBE_MAC_CHAIN,
 * 2 independent 8-word steps, i.e. 32 multiply-adds).  A checksum per block is
 * written to out[blockIdx] (device memory, `blocks` words) so nothing is
 * optimised away.  *ops_per_thread receives the multiply-adds each thread
 * performs.  Errors: BN_EINVAL (null pointers, zero sizes, threads > 1024 or
 * not a multiple of 32, unknown kind), BN_ECUDA. */
bn_status bn_probe_int_throughput(int kind, uint32_t blocks, uint32_t threads, uint32_t iters,
                                  uint32_t *out, uint64_t *ops_per_thread, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BN_GB300_PROBE_H */
