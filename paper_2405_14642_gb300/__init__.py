"""Batched exact addition and multiplication of midsize unsigned integers on
one NVIDIA GB300 (sm_103a), after Oancea & Watt, "GPU Implementations for
Midsize Integer Addition and Multiplication" (arXiv 2405.14642).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/bn.h``); this package is its thin ctypes binding.  Operations:

* :func:`bn_add` - addition by a carry-propagation scan (Section 2);
* :func:`bn_mul` - multiplication by the fastest method for the sizes;
* :func:`bn_mul_quad` - classical multiplication with a load-balanced
  per-thread partition of the result (Section 3);
* :func:`bn_mul_ntt` - multiplication through a number-theoretic transform
  over "good" primes, one 64-bit prime with 16-bit digits or two primes with
  32-bit digits and CRT recombination (Section 4); :func:`bn_mul_ntt3` -
  the same over three 32-bit primes;
* :func:`bn_mul_quad_tc` - the classical product's column sums computed on
  bytes as an exact fp16 contraction on the tensor cores;
* :func:`bn_mul_low`, :func:`bn_poly`, :func:`bn_add6` - same-length
  (mod 2^(32 n)) product and the two fused programs of Section 6;
* :class:`Plan` - the plan object of the C ABI (device and host-buffer forms);
* :class:`Batch` - many operations of mixed sizes and kinds as one CUDA graph;
* :class:`Server` - a serving loop that batches device-resident requests
  continuously as they arrive.
"""
from ._binding import (COMPLETION_DTYPE, REQUEST_DTYPE, Server, device_to_host,
                       BATCH_ITEM_DTYPE, BN_BATCH_AUTOTUNE, BN_BATCH_PLAIN, BN_BATCH_PLAIN_CLASSES,
                       BN_OP_MUL_AUTO, Batch,
                       BN_ADD_MAX_LIMBS, BN_MUL_MAX_LIMBS, BN_OP_ADD, BN_OP_MUL_NTT64,
                       BN_OP_MUL_NTT_CRT, BN_OP_MUL_NTT3, BN_OP_MUL_QUAD, BN_OP_MUL_QUAD_TC, BN_ETIMEOUT, BnError, Plan, bn_add,
                       bn_mul, bn_mul_ntt, bn_mul_ntt3, bn_mul_quad_tc, bn_tc_check, bn_tc_wait_selftest,
                       bn_add6, bn_mul_low, bn_mul_ntt_noalloc, bn_mul_quad, bn_poly,
                       bn_probe_int_throughput, bn_probe_mma_throughput, library_path, load)

__all__ = ["bn_add", "bn_mul_quad", "bn_mul_ntt", "Plan", "BnError", "load", "library_path",
           "BN_OP_ADD", "BN_OP_MUL_QUAD", "BN_OP_MUL_NTT64", "BN_OP_MUL_NTT_CRT",
           "BN_ADD_MAX_LIMBS", "BN_MUL_MAX_LIMBS", "bn_probe_int_throughput", "bn_probe_mma_throughput",
           "bn_mul_ntt_noalloc", "Batch", "BATCH_ITEM_DTYPE", "BN_BATCH_AUTOTUNE", "BN_BATCH_PLAIN", "BN_BATCH_PLAIN_CLASSES",
           "BN_OP_MUL_AUTO", "Server", "REQUEST_DTYPE", "COMPLETION_DTYPE", "device_to_host",
           "bn_mul_low", "bn_poly", "bn_add6", "bn_mul_ntt3", "BN_OP_MUL_NTT3", "bn_mul",
           "bn_mul_quad_tc", "bn_tc_check", "bn_tc_wait_selftest", "BN_OP_MUL_QUAD_TC",
           "BN_ETIMEOUT"]
