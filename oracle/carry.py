"""The paper's carry-propagation operator and scan-based addition (Section 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Small Python-int cases.

Section 2 turns big-integer addition into three data-parallel steps:

1. a map producing, per word, the partial sum ``p_i = a_i + b_i mod 2^w`` and
   two flags: ``ov_i`` (the word addition overflowed, ``p_i < a_i``) and
   ``mx_i`` (the partial sum is the largest word, ``p_i == 2^w - 1``);
2. an exclusive scan of the flag pairs with an associative carry operator
   whose neutral element is ``(ov, mx) = (False, True)``;
3. a map adding each scanned carry into its partial sum.

The operator composes an accumulated prefix ``(ov1, mx1)`` with the next word
``(ov2, mx2)``: a carry leaves the combined range if the next word overflowed by
itself, or if it is the largest word and a carry arrives from the prefix; the
combined range is all-largest-words only if both parts are.

Two encodings appear in the paper: the boolean pair, and a packed u32 with the
overflow flag in bit 0 and the largest-word flag in bit 1 (neutral value 2).
For several instances sharing one scan, bit 2 marks the first word of each
instance and the lifted operator restarts the carry there (a segmented scan).

The exclusive scan is read as the standard one: ``out_0`` is the neutral
element and ``out_i`` folds elements ``0 .. i-1`` (the printed index list of
the definition is garbled).

Segmented reading.  Section 2's batched form applies a plain exclusive scan
with the lifted operator.  Taken literally, the output at the first word of an
instance is the fold of everything before it, i.e. the previous instance's
carry-out, which would leak into the next sum.  A segmented exclusive scan is
read here by its definition, an exclusive scan of each segment on its own: the
output at a segment start is the neutral element.  The tests pin both the leak
of the literal form and the exactness of this reading.
"""
from __future__ import annotations

from typing import Callable, Iterable, List, Sequence, Tuple

Flags = Tuple[bool, bool]
NEUTRAL_PAIR: Flags = (False, True)
NEUTRAL_PACKED = 2


def carry_pair(x: Flags, y: Flags) -> Flags:
    """Boolean-pair carry operator, Section 2."""
    ov_x, mx_x = x
    ov_y, mx_y = y
    return (ov_y or (ov_x and mx_y), mx_x and mx_y)


def pack(flags: Flags, segment_start: bool = False) -> int:
    ov, mx = flags
    return int(ov) | (int(mx) << 1) | (int(segment_start) << 2)


def unpack(c: int) -> Flags:
    return (bool(c & 1), bool(c & 2))


def carry_packed(x: int, y: int) -> int:
    """Packed form of the operator on bits 0 (overflow) and 1 (largest word)."""
    mx = x & y & 2
    ov = (y | (x & (y >> 1))) & 1
    return mx | ov


def carry_segmented(x: int, y: int) -> int:
    """Packed operator lifted to segments: bit 2 of ``y`` restarts the carry."""
    if y & 4:
        return y
    return carry_packed(x, y) | ((x | y) & 4)


def exclusive_scan(op: Callable, neutral, xs: Sequence) -> List:
    """out[0] = neutral, out[i] = xs[0] op ... op xs[i-1] (sequential fold)."""
    out, acc = [], neutral
    for x in xs:
        out.append(acc)
        acc = op(acc, x)
    return out


def segmented_exclusive_scan(xs: Sequence[int]) -> List[int]:
    """Exclusive scan of each segment on its own (segments start at bit 2)."""
    out, acc = [], NEUTRAL_PACKED
    for x in xs:
        if x & 4:
            acc = NEUTRAL_PACKED | 4
        out.append(acc)
        acc = carry_segmented(acc, x)
    return out


def inclusive_total(op: Callable, neutral, xs: Iterable):
    acc = neutral
    for x in xs:
        acc = op(acc, x)
    return acc


def add_by_scan(a: Sequence[int], b: Sequence[int], w: int = 32) -> List[int]:
    """a + b as len(a)+1 words of w bits, by the three steps of Section 2.

    ``a`` and ``b`` have the same number of words.  The extra top word is the
    carry out of the whole range (the overflow flag of the inclusive fold).
    """
    if len(a) != len(b):
        raise ValueError("equal word counts expected")
    top = (1 << w) - 1
    partial, flags = [], []
    for ai, bi in zip(a, b):                      # step 1: map
        p = (ai + bi) & top
        partial.append(p)
        flags.append((p < ai, p == top))
    carries = exclusive_scan(carry_pair, NEUTRAL_PAIR, flags)  # step 2: scan
    result = [(p + int(c[0])) & top for p, c in zip(partial, carries)]  # step 3
    result.append(int(inclusive_total(carry_pair, NEUTRAL_PAIR, flags)[0]))
    return result


def add_batch_segmented(a_insts: Sequence[Sequence[int]],
                        b_insts: Sequence[Sequence[int]], w: int = 32,
                        literal: bool = False) -> List[List[int]]:
    """Several equal-length additions in ONE segmented scan (Section 2, IPB > 1).

    Returns each instance's sum with its carry word appended, so the results
    compare directly with :func:`add_by_scan` and the C oracle.  ``literal``
    uses the plain exclusive scan with the lifted operator (see the module
    notes); it is kept only to show that form leaking carries.
    """
    top = (1 << w) - 1
    m = len(a_insts[0])
    partial, packed = [], []
    for a, b in zip(a_insts, b_insts):
        if len(a) != m or len(b) != m:
            raise ValueError("equal word counts expected")
        for i, (ai, bi) in enumerate(zip(a, b)):
            p = (ai + bi) & top
            partial.append(p)
            packed.append(pack((p < ai, p == top), segment_start=(i == 0)))
    if literal:
        carries = exclusive_scan(carry_segmented, NEUTRAL_PACKED, packed)
    else:
        carries = segmented_exclusive_scan(packed)
    out = []
    for k in range(len(a_insts)):
        lo, hi = k * m, (k + 1) * m
        words = [(partial[i] + (carries[i] & 1)) & top for i in range(lo, hi)]
        total = inclusive_total(carry_segmented, NEUTRAL_PACKED, packed[lo:hi])
        words.append(total & 1)
        out.append(words)
    return out
