"""Checks that pin the oracle to facts other than itself.

Each ``check_*`` takes an object with the oracle's ``add/sub/mul/mod_u64``
methods and raises ``AssertionError`` on the first disagreement, so the same
checks run against the real oracle and against deliberately broken copies
(``test_oracle_mutants.py``), showing that a plausible mistake fails one of them.

The independent facts:
* CPython's own big-integer arithmetic (a separate implementation);
* closed forms listed in ``golden/closed_forms.txt``;
* brute force over an alphabet of boundary limb values;
* algebraic invariants (commutativity, (a+b)-b = a, distributivity, residues
  modulo 61/62-bit primes).
"""
from __future__ import annotations

import itertools
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).resolve().parent / "golden"
MASK32 = (1 << 32) - 1


def to_int(limbs) -> int:
    return int.from_bytes(np.ascontiguousarray(limbs, dtype="<u4").tobytes(), "little")


def from_int(v: int, n: int) -> np.ndarray:
    return np.frombuffer(v.to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def rand_batch(rng, batch, n):
    return rng.integers(0, 1 << 32, size=(batch, n), dtype=np.uint64).astype(np.uint32)


def check_python_ints(orc, seed=1):
    rng = np.random.default_rng(seed)
    shapes = [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (7, 5), (31, 33), (64, 64),
              (100, 37), (128, 128), (129, 255), (300, 300)]
    for na, nb in shapes:
        a, b = rand_batch(rng, 6, na), rand_batch(rng, 6, nb)
        s, p = orc.add(a, b), orc.mul(a, b)
        for i in range(6):
            x, y = to_int(a[i]), to_int(b[i])
            assert to_int(s[i]) == x + y, ("add", na, nb, i)
            assert to_int(p[i]) == x * y, ("mul", na, nb, i)


def _closed_form(form: str, L: int):
    ones = np.full(L, MASK32, np.uint32)
    if form == "sq_allones":
        want = np.zeros(2 * L, np.uint32)
        want[0] = 1
        want[L] = 0xFFFFFFFE
        want[L + 1:] = MASK32
        return "mul", ones, ones, want
    if form == "dbl_allones":
        want = np.full(L + 1, MASK32, np.uint32)
        want[0] = 0xFFFFFFFE
        want[L] = 1
        return "add", ones, ones, want
    if form == "inc_allones":
        one = np.zeros(L, np.uint32)
        one[0] = 1
        want = np.zeros(L + 1, np.uint32)
        want[L] = 1
        return "add", ones, one, want
    raise ValueError(form)


def closed_form_cases():
    for line in (GOLDEN / "closed_forms.txt").read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        form, L = line.split()
        yield (form, int(L)) + _closed_form(form, int(L))


def check_closed_forms(orc):
    for form, L, op, a, b, want in closed_form_cases():
        got = (orc.mul if op == "mul" else orc.add)(a[None], b[None])[0]
        # The identity itself, restated with Python ints, guards the table.
        x, y = to_int(a), to_int(b)
        assert to_int(want) == (x * y if op == "mul" else x + y), (form, L)
        assert np.array_equal(got, want), (form, L)
    # 2^i * 2^j = 2^(i+j); 0 * x = 0; 1 * x = x.
    n = 9
    for i, j in [(0, 0), (31, 1), (32, 32), (100, 187), (287, 287)]:
        a, b = from_int(1 << i, n), from_int(1 << j, n)
        assert to_int(orc.mul(a[None], b[None])[0]) == 1 << (i + j), (i, j)
    x = rand_batch(np.random.default_rng(5), 1, n)
    zero, one = np.zeros((1, n), np.uint32), from_int(1, n)[None]
    assert not orc.mul(zero, x).any()
    assert to_int(orc.mul(one, x)[0]) == to_int(x[0])


ALPHABET = [0, 1, 2, 1 << 31, MASK32 - 1, MASK32, 0x9E3779B9]


def check_bruteforce(orc, max_limbs=2):
    for n in range(1, max_limbs + 1):
        vals = list(itertools.product(ALPHABET, repeat=n))
        a = np.array([v for v in vals for _ in vals], np.uint32)
        b = np.array([w for _ in vals for w in vals], np.uint32)
        s, p = orc.add(a, b), orc.mul(a, b)
        for i in range(a.shape[0]):
            x, y = to_int(a[i]), to_int(b[i])
            assert to_int(s[i]) == x + y, ("add", a[i], b[i])
            assert to_int(p[i]) == x * y, ("mul", a[i], b[i])
    # Mixed lengths: 1 x 3 and 3 x 1 over the alphabet.
    for na, nb in [(1, 3), (3, 1)]:
        av = list(itertools.product(ALPHABET[:4], repeat=na))
        bv = list(itertools.product(ALPHABET[3:], repeat=nb))
        a = np.array([v for v in av for _ in bv], np.uint32)
        b = np.array([w for _ in av for w in bv], np.uint32)
        s, p = orc.add(a, b), orc.mul(a, b)
        for i in range(a.shape[0]):
            x, y = to_int(a[i]), to_int(b[i])
            assert to_int(s[i]) == x + y and to_int(p[i]) == x * y


# Primes near 2^61 / 2^62 for residue checks (primality is verified in a test).
RESIDUE_PRIMES = [(1 << 61) - 1, 4179340454199820289, 2305843009213693921, 4611686018427387847]


def check_invariants(orc, seed=2):
    rng = np.random.default_rng(seed)
    for na, nb in [(17, 17), (40, 9), (128, 128), (257, 64)]:
        a, b = rand_batch(rng, 4, na), rand_batch(rng, 4, nb)
        ab, ba = orc.mul(a, b), orc.mul(b, a)
        assert np.array_equal(ab, ba), ("commutativity", na, nb)
        s = orc.add(a, b)                               # (a + b) - b = a
        d, borrow = orc.sub(s, b)
        assert not borrow.any()
        assert np.array_equal(d[:, :na], a) and not d[:, na:].any(), ("sub", na, nb)
        c = rand_batch(rng, 4, nb)                      # a (b + c) = a b + a c
        lhs = orc.mul(a, orc.add(b, c))
        rhs = orc.add(orc.mul(a, b), orc.mul(a, c))
        assert np.array_equal(lhs[:, : na + nb + 1], rhs[:, : na + nb + 1]), ("distrib", na, nb)
        for i in range(4):
            for q in RESIDUE_PRIMES:
                ra, rb = orc.mod_u64(a[i], q), orc.mod_u64(b[i], q)
                assert orc.mod_u64(ab[i], q) == ra * rb % q, ("residue", q)
                assert ra == to_int(a[i]) % q
    # Results do not depend on how the batch is split across threads.
    a, b = rand_batch(rng, 37, 65), rand_batch(rng, 37, 33)
    assert np.array_equal(orc.mul(a, b, threads=1), orc.mul(a, b, threads=5))
    assert np.array_equal(orc.add(a, b, threads=1), orc.add(a, b, threads=7))


ALL_CHECKS = (check_python_ints, check_closed_forms, check_bruteforce, check_invariants)
