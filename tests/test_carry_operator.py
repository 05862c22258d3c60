"""Pins of the Section 2 carry operator and the scan-based addition (no GPU)."""
import itertools

import numpy as np

from oracle import carry
import pins

STATES = list(itertools.product([False, True], repeat=2))


def test_packed_form_matches_pair_form():
    for x, y in itertools.product(STATES, STATES):
        assert carry.unpack(carry.carry_packed(carry.pack(x), carry.pack(y))) == carry.carry_pair(x, y)


def test_neutral_element():
    for x in STATES:
        assert carry.carry_pair(carry.NEUTRAL_PAIR, x) == x
        assert carry.carry_pair(x, carry.NEUTRAL_PAIR) == x
        assert carry.carry_packed(carry.NEUTRAL_PACKED, carry.pack(x)) == carry.pack(x)
        assert carry.carry_packed(carry.pack(x), carry.NEUTRAL_PACKED) == carry.pack(x)


def test_associativity_exhaustive():
    for x, y, z in itertools.product(STATES, repeat=3):
        assert carry.carry_pair(carry.carry_pair(x, y), z) == carry.carry_pair(x, carry.carry_pair(y, z))
    seg = [carry.pack(s, st) for s in STATES for st in (False, True)]
    for x, y, z in itertools.product(seg, repeat=3):
        assert carry.carry_segmented(carry.carry_segmented(x, y), z) == \
            carry.carry_segmented(x, carry.carry_segmented(y, z))


def test_one_word_never_overflows_and_is_largest():
    # ov = (p < a) and mx = (p == max) exclude each other for a single word,
    # exhaustively in base 2^4.
    for a, b in itertools.product(range(16), repeat=2):
        p = (a + b) & 15
        assert not (p < a and p == 15)


def test_scan_add_exhaustive_base4():
    """Every pair of 4-word numbers in base 2^2 (all 3^4 flag vectors occur)."""
    for x in range(256):
        xa = [(x >> (2 * i)) & 3 for i in range(4)]
        for y in range(256):
            ya = [(y >> (2 * i)) & 3 for i in range(4)]
            got = carry.add_by_scan(xa, ya, w=2)
            assert sum(v << (2 * i) for i, v in enumerate(got)) == x + y


def test_scan_add_matches_c_oracle(oracle_mod):
    rng = np.random.default_rng(7)
    cases = [pins.rand_batch(rng, 3, 40) for _ in range(2)]
    ones = np.full((1, 40), 0xFFFFFFFF, np.uint32)
    one = np.zeros((1, 40), np.uint32)
    one[0, 0] = 1
    for a, b in [tuple(cases), (ones, one), (ones, ones)]:
        want = oracle_mod.add(a, b)
        for i in range(a.shape[0]):
            assert carry.add_by_scan(list(map(int, a[i])), list(map(int, b[i]))) == list(map(int, want[i]))


def test_segmented_scan_equals_separate_scans(oracle_mod):
    rng = np.random.default_rng(8)
    a, b = pins.rand_batch(rng, 8, 12), pins.rand_batch(rng, 8, 12)
    a[2] = 0xFFFFFFFF
    b[2] = 0
    b[2, 0] = 1                      # a full carry chain that must not leak
    a[3] = 0xFFFFFFFF
    b[3] = 0                         # ...into an all-largest neighbour
    got = carry.add_batch_segmented([list(map(int, r)) for r in a], [list(map(int, r)) for r in b])
    want = oracle_mod.add(a, b)
    assert got == [list(map(int, r)) for r in want]


def test_literal_segmented_form_leaks_carry(oracle_mod):
    """The batched form read literally (plain exclusive scan with the lifted
    operator) adds instance k's carry-out into instance k+1's first word."""
    a = np.array([[0xFFFFFFFF, 0xFFFFFFFF], [5, 6]], np.uint32)
    b = np.array([[1, 0], [7, 8]], np.uint32)
    want = [list(map(int, r)) for r in oracle_mod.add(a, b)]
    lists = ([list(map(int, r)) for r in a], [list(map(int, r)) for r in b])
    assert carry.add_batch_segmented(*lists) == want
    leaked = carry.add_batch_segmented(*lists, literal=True)
    assert leaked[1][0] == want[1][0] + 1
