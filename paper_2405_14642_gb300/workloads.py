"""Seeded synthetic operand batches shaped like the paper's workloads.

This module only draws random limbs and stamps structured edge-case values; it
performs none of the method's arithmetic, so both the GPU tests and the CPU
oracle checks can take their inputs from it.

The paper's experiments (Section 6.1) use synthetic batches with
``NumBits * NumInsts = 2^32`` over sizes 2^11 .. 2^18 bits and do not state the
value distribution.  The stand-ins here:

* limbs uniform over u32 from ``numpy.random.PCG64(seed)``;
* seed = ``0xB16 + 1000 * workload_index + size_index``;
* "edge" batches replace every instance ``i`` with ``i % 20 == 19`` (5%) by one of
  five structured cases, cycling by ``(i // 20) % 5``:

  0. a = b = all-ones (longest carry chains, largest products);
  1. a = all-ones, b = 1 (a carry through every limb of the sum);
  2. a = 0;
  3. a and b single-limb values (limb 0 random, the rest zero);
  4. a = all-ones, b uniform.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

SEED_BASE = 0xB16
ALL_ONES = np.uint32(0xFFFFFFFF)

# Integer sizes of the size sweep, in bits (2^10 .. 2^18).
SWEEP_BITS: Tuple[int, ...] = tuple(1 << e for e in range(10, 19))
# Sizes where the transform-based products are measured (2^14 .. 2^18 bits).
NTT_BITS: Tuple[int, ...] = tuple(1 << e for e in range(14, 19))
# Operand bytes per side in the size sweep: 64 MiB.
SWEEP_SIDE_BYTES = 64 << 20


def seed_for(workload_index: int, size_index: int = 0) -> int:
    return SEED_BASE + 1000 * workload_index + size_index


def uniform_limbs(batch: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """(batch, n) uniform u32 limbs."""
    return rng.integers(0, 1 << 32, size=(batch, n), dtype=np.uint64).astype(np.uint32)


def stamp_edge_cases(a: np.ndarray, b: np.ndarray, rng: np.random.Generator) -> None:
    """Overwrite every 20th instance (i % 20 == 19) with the five edge cases."""
    batch = a.shape[0]
    for i in range(19, batch, 20):
        kind = (i // 20) % 5
        if kind == 0:
            a[i] = ALL_ONES
            b[i] = ALL_ONES
        elif kind == 1:
            a[i] = ALL_ONES
            b[i] = 0
            b[i, 0] = 1
        elif kind == 2:
            a[i] = 0
        elif kind == 3:
            a[i] = 0
            b[i] = 0
            a[i, 0] = rng.integers(0, 1 << 32, dtype=np.uint64)
            b[i, 0] = rng.integers(0, 1 << 32, dtype=np.uint64)
        else:
            a[i] = ALL_ONES


def pair_batch(batch: int, na: int, nb: int | None = None, seed: int = SEED_BASE,
               edges: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """Seeded operand pair batch: a (batch, na), b (batch, nb)."""
    nb = na if nb is None else nb
    rng = np.random.Generator(np.random.PCG64(seed))
    a = uniform_limbs(batch, na, rng)
    b = uniform_limbs(batch, nb, rng)
    if edges:
        stamp_edge_cases(a, b, rng)
    return a, b


@dataclass(frozen=True)
class SweepPoint:
    bits: int
    limbs: int
    batch: int
    seed: int


def sweep_points(bits_list=SWEEP_BITS, side_bytes: int = SWEEP_SIDE_BYTES,
                 workload_index: int = 1) -> List[SweepPoint]:
    """Size sweep: batch chosen so each side holds ``side_bytes`` of limbs."""
    pts = []
    for idx, bits in enumerate(bits_list):
        n = bits // 32
        pts.append(SweepPoint(bits, n, side_bytes // (4 * n), seed_for(workload_index, idx)))
    return pts


def tiny_workload() -> Tuple[np.ndarray, np.ndarray]:
    """4096 pairs of 4096-bit integers (128 limbs) with 5% edge cases."""
    return pair_batch(4096, 128, seed=seed_for(0), edges=True)


# Op codes of include/bn.h used by mixed workloads.
OP_ADD, OP_MUL_AUTO = 0, 4
MIXED_ITEM_DTYPE = np.dtype([("op", "<u4"), ("na", "<u4"), ("nb", "<u4"), ("reserved", "<u4"),
                             ("a_offset", "<u8"), ("b_offset", "<u8"), ("c_offset", "<u8")])


def log_uniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Integer limb counts with log-uniform distribution on [lo, hi]."""
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.rint(x), lo, hi).astype(np.uint32)


def mixed_workload(count: int, seed: int, lo: int = 32, hi: int = 8192, mul_frac: float = 0.7,
                   edges: bool = True, mul_op: int = OP_MUL_AUTO):
    """Mixed batch: `count` operations, a fraction `mul_frac` products (op
    `mul_op`) and the rest additions, operand limb counts log-uniform in
    [lo, hi] independently for a and b, limbs uniform; with `edges`, every
    20th item (i % 20 == 19) gets one of the five edge cases of the sweep.

    Returns (items, a_flat, b_flat, c_limbs): items of MIXED_ITEM_DTYPE with
    offsets into the flat operand arrays and a flat result array of c_limbs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items = np.zeros(count, MIXED_ITEM_DTYPE)
    is_mul = rng.random(count) < mul_frac
    items["op"] = np.where(is_mul, mul_op, OP_ADD)
    items["na"] = log_uniform_sizes(rng, count, lo, hi)
    items["nb"] = log_uniform_sizes(rng, count, lo, hi)
    na = items["na"].astype(np.uint64)
    nb = items["nb"].astype(np.uint64)
    nout = np.where(is_mul, na + nb, np.maximum(na, nb) + 1).astype(np.uint64)
    items["a_offset"] = np.concatenate(([0], np.cumsum(na)[:-1])) if count else []
    items["b_offset"] = np.concatenate(([0], np.cumsum(nb)[:-1])) if count else []
    items["c_offset"] = np.concatenate(([0], np.cumsum(nout)[:-1])) if count else []
    a = uniform_limbs(1, int(na.sum()), rng)[0] if count else np.zeros(0, np.uint32)
    b = uniform_limbs(1, int(nb.sum()), rng)[0] if count else np.zeros(0, np.uint32)
    if edges:
        for i in range(19, count, 20):
            ao, bo = int(items["a_offset"][i]), int(items["b_offset"][i])
            ra = a[ao:ao + int(na[i])]
            rb = b[bo:bo + int(nb[i])]
            kind = (i // 20) % 5
            if kind == 0:
                ra[:] = ALL_ONES
                rb[:] = ALL_ONES
            elif kind == 1:
                ra[:] = ALL_ONES
                rb[:] = 0
                rb[0] = 1
            elif kind == 2:
                ra[:] = 0
            elif kind == 3:
                ra[1:] = 0
                rb[1:] = 0
            else:
                ra[:] = ALL_ONES
    return items, a, b, int(nout.sum())

