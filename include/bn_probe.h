/*
 * bn_probe.h - measurement helpers for the integer-multiply and tensor-core rooflines.
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

/* Enqueue the tensor-core chain probe: `ctas` CTAs (one per SM: each holds
 * 130 KB of shared memory) each issue `iters` MMAs (tcgen05.mma kind::f16,
 * M = 128, K = 16, N = n, operands in shared memory at windows that move with
 * every MMA, as the tensor-core schoolbook's do) from one thread, round-robin
 * over `chains` accumulators of n tensor-memory columns, each restarted
 * (accumulate = 0) every `chain_len` of its MMAs.  Timing it gives the SM
 * clocks per MMA of a given number of independent accumulation chains.  The
 * operands are zero.  *status (device memory) is set to 1 if the wait for the
 * MMAs timed out (after 2 s; the kernel then frees its tensor memory and
 * returns).  Errors: BN_EINVAL (null status, zero sizes, n not a multiple of
 * 16 in [16, 256], n * chains > 512), BN_ECUDA. */
bn_status bn_probe_mma_throughput(uint32_t n, uint32_t chains, uint32_t chain_len, uint32_t iters,
                                  uint32_t ctas, uint32_t *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BN_GB300_PROBE_H */
