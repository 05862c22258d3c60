"""CPU model of the schoolbook's lane form (one product per thread): the
windows of Q = 8 columns in order, each split into the falling triangle, the
full blocks and the rising triangle (Section 3, Eq. (1), Fig. 3's columns),
with the kernel's block bounds, chain lengths and pending-carry words.

It checks the decomposition, not the oracle: every word product a_i b_j with
i < na, j < nb is taken exactly once and no padding product is; the Q + 2
word accumulator (with its separately counted carries) never overflows; the
window words stored equal those of a * b, computed with Python integers; and
the staging's stepped (row, offset) pairs give every unit exactly once.
Planted slips (a block bound off by one, a rising
chain one word short, the carry-in dropped) must fail.
"""
import random

import pytest

Q = 8
W32 = (1 << 32) - 1


def roundup(x, m):
    return (x + m - 1) // m * m


def lane_product(a, b, slip=None):
    """The kernel's window loop over Python-int words; returns the stored
    words and the multiset of (i, j) pairs multiplied."""
    na, nb = len(a), len(b)
    if na < nb:
        a, b, na, nb = b, a, nb, na
    nap, nbp, nout = roundup(na, Q), roundup(nb, Q), na + nb
    A = a + [0] * (nap - na)
    B = b + [0] * (nbp - nb)
    NA, NB, KW = nap // Q, nbp // Q, (nout + Q - 1) // Q
    pairs = []
    out = []
    acc = [0] * (Q + 2)

    def chain(words, start, a_word, ws, half, carry_to):
        """words[start + q] += half of a_word * ws[q] with a carry chain; the
        chain's carry out is returned (the kernel adds it to `carry_to`)."""
        c = 0
        for q, w in enumerate(ws):
            prod = a_word * w
            v = (prod & W32) if half == "lo" else (prod >> 32)
            t = words[start + q] + v + c
            words[start + q] = t & W32
            c = t >> 32
        return c

    for K in range(KW):
        carry = (acc[Q], acc[Q + 1]) if slip != "carry_in" else (0, 0)
        acc = [carry[0], carry[1]] + [0] * Q
        cnt = 0
        if K >= NB:                                  # falling triangle: B block NB-1's top words
            I = K - NB
            lo = B[(NB - 1) * Q:NB * Q]
            pend = [0] * (Q + 1)
            for s in range(1, Q):
                ai = I * Q + s
                ws = lo[Q - s:]
                pairs += [(ai, (NB - 1) * Q + Q - s + q) for q in range(s)]
                pend[s] += chain(acc, 0, A[ai], ws, "lo", None)
                pend[s + 1] += chain(acc, 1, A[ai], ws, "hi", None)
            c = 0
            for w in range(1, Q + 2):
                t = acc[w] + (pend[w] if w <= Q else 0) + c
                acc[w], c = t & W32, t >> 32
            assert c == 0, "accumulator overflow"
        i0 = K + 1 - NB if K + 1 > NB else 0
        i1 = K if K < NA else NA
        if slip == "full_bound":
            i1 = min(i1 + 1, NA)
        for I in range(i0, i1):                     # full blocks: B blocks J-1 and J
            J = K - I
            for s in range(Q):
                ai = I * Q + s
                ws = [B[J * Q - s + q] for q in range(Q)]
                pairs += [(ai, J * Q - s + q) for q in range(Q)]
                cnt += chain(acc, 0, A[ai], ws, "lo", None)
                acc[Q + 1] += chain(acc, 1, A[ai], ws, "hi", None)
        if K < NA:                                  # rising triangle: B block 0's low words
            for s in range(Q):
                ai = K * Q + s
                m = Q - s - (1 if slip == "rising_short" and s == 3 else 0)
                ws = B[:m]
                pairs += [(ai, q) for q in range(m)]
                cnt += chain(acc, s, A[ai], ws, "lo", None)
                acc[Q + 1] += chain(acc, s + 1, A[ai], ws, "hi", None)
        t = acc[Q] + cnt                            # fold_count
        acc[Q], acc[Q + 1] = t & W32, acc[Q + 1] + (t >> 32)
        assert all(0 <= w <= W32 for w in acc), "accumulator word out of range"
        out += acc[:Q]
    assert acc[Q] == 0 and acc[Q + 1] == 0, "carry out of the last window"
    return out[:nout], out[nout:], pairs, (na, nb)


def value(words):
    return sum(w << (32 * i) for i, w in enumerate(words))


def words_of(x, n):
    return [(x >> (32 * i)) & W32 for i in range(n)]


SIZES = [(1, 1), (1, 8), (3, 2), (7, 7), (8, 8), (9, 1), (16, 9), (32, 32), (33, 31), (40, 24),
         (64, 64), (64, 1), (100, 3), (128, 128), (127, 65)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_lane_windows_cover_each_pair_once(na, nb):
    rng = random.Random(na * 131 + nb)
    for kind in ("max", "rand"):
        a = [W32] * na if kind == "max" else [rng.getrandbits(32) for _ in range(na)]
        b = [W32] * nb if kind == "max" else [rng.getrandbits(32) for _ in range(nb)]
        got, beyond, pairs, (ha, hb) = lane_product(a, b)
        assert got == words_of(value(a) * value(b), na + nb)
        assert all(w == 0 for w in beyond)
        real = [(i, j) for i, j in pairs if i < ha and j < hb]
        assert sorted(real) == [(i, j) for i in range(ha) for j in range(hb)]
        # padding products only where the operand is not a multiple of Q
        if ha % Q == 0 and hb % Q == 0:
            assert len(pairs) == ha * hb


@pytest.mark.parametrize("slip", ["full_bound", "rising_short", "carry_in"])
def test_lane_planted_slips_fail(slip):
    a, b = [W32] * 32, [W32] * 32
    with pytest.raises(AssertionError):
        got, beyond, pairs, _ = lane_product(a, b, slip=slip)
        assert got == words_of(value(a) * value(b), 64)
        assert sorted(pairs) == [(i, j) for i in range(32) for j in range(32)]


def test_staging_steps_cover_each_unit_once():
    """The warp's staging: lane l takes units x = l, l + 32, ... of an
    nrows x d block and finds (row, unit in row) by stepping (r, o) with x,
    never dividing: every unit lands once, at its own row and offset."""
    for d in list(range(1, 40)) + [64, 96, 128]:
        for nrows in (1, 2, 7, 31, 32):
            total = nrows * d
            seen = []
            for lane in range(32):
                sr, so = 32 // d, 32 % d
                r, o = lane // d, lane % d
                for x in range(lane, total, 32):
                    assert (r, o) == divmod(x, d)
                    seen.append((r, o))
                    r, o = r + sr, o + so
                    if o >= d:
                        r, o = r + 1, o - d
            assert sorted(seen) == [(r, o) for r in range(nrows) for o in range(d)]


@pytest.mark.parametrize("na,nb", [(1, 1), (32, 32), (64, 64), (128, 128), (100, 3)])
def test_lane_stride_is_an_odd_number_of_units(na, nb):
    nap, nbp = roundup(na, Q), roundup(nb, Q)
    s = roundup(nap + nbp, 4)
    if (s // 4) % 2 == 0:
        s += 4
    assert s >= nap + nbp and s % 4 == 0 and (s // 4) % 2 == 1
    # eight consecutive lanes' 16-byte reads at the same offset hit eight distinct bank groups
    assert len({(l * s // 4) % 8 for l in range(8)}) == 8
