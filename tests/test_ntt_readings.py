"""Pins of the Section 4 prime fields and transform readings (no GPU)."""
from pathlib import Path

import numpy as np
import pytest

from oracle import ntt
import pins
from test_oracle_pins import is_probable_prime

GOLDEN = Path(__file__).resolve().parent / "golden" / "prime_fields.txt"
FIELDS = [ntt.PRIME_FIELD_32, ntt.PRIME_FIELD_64, ntt.PRIME_FIELD_CRT2, *ntt.PRIME_FIELDS_3X32]


def golden_fields():
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, p, k, n, g = line.split()
            yield name, int(p), int(k), int(n), int(g)


def test_printed_fields_match_module_constants():
    got = {(f.name, f.p, f.k, f.n, f.g) for f in (ntt.PRIME_FIELD_32, ntt.PRIME_FIELD_64)}
    assert got == set(golden_fields())


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_field_shape_primality_and_root_order(field):
    assert field.p == field.k * (1 << field.n) + 1
    assert is_probable_prime(field.p)
    assert pow(field.g, 1 << field.n, field.p) == 1
    assert pow(field.g, 1 << (field.n - 1), field.p) != 1   # order exactly 2^n


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_root_search_and_derived_roots(field):
    g = ntt.search_root(field.p, field.k, field.n)
    if field is ntt.PRIME_FIELD_CRT2 or field in ntt.PRIME_FIELDS_3X32:
        assert g == field.g                  # the chosen root is the search's first hit
    assert pow(g, 1 << field.n, field.p) == 1 and pow(g, 1 << (field.n - 1), field.p) != 1
    for m in [2, 4, 1024, 1 << 15]:
        w = field.root(m)
        assert pow(w, m, field.p) == 1
        assert pow(w, m // 2, field.p) == field.p - 1
    tab = ntt.powers(field.root(16), 16, field.p)
    assert tab == [pow(field.root(16), j, field.p) for j in range(16)]


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_fast_transform_equals_definition(field):
    rng = np.random.default_rng(4)
    for m in [1, 2, 4, 8, 32]:
        x = [int(v) % field.p for v in rng.integers(0, 1 << 62, size=m, dtype=np.uint64)]
        w = field.root(m) if m > 1 else 1
        assert ntt.ntt(x, w, field.p) == ntt.dft(x, w, field.p)
        assert ntt.intt(ntt.ntt(x, w, field.p), w, field.p) == x
    m = 16
    w = field.root(m)
    for i in range(m):
        delta = [0] * m
        delta[i] = 1
        assert ntt.ntt(delta, w, field.p) == [pow(w, i * j, field.p) for j in range(m)]


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_convolution_theorem(field):
    rng = np.random.default_rng(5)
    for m in [4, 16, 64]:
        x = [int(v) for v in rng.integers(0, 1 << 20, size=m)]
        y = [int(v) for v in rng.integers(0, 1 << 20, size=m)]
        w = field.root(m)
        spec = [u * v % field.p for u, v in zip(ntt.ntt(x, w, field.p), ntt.ntt(y, w, field.p))]
        assert ntt.intt(spec, w, field.p) == ntt.cyclic_convolution(x, y, field.p)


def _cases(rng, n):
    a, b = pins.rand_batch(rng, 2, n), pins.rand_batch(rng, 2, n)
    a[1] = 0xFFFFFFFF
    b[1] = 0xFFFFFFFF
    return a, b


@pytest.mark.parametrize("n", [1, 3, 32, 128])
def test_single_prime_16bit_digits_exact(oracle_mod, n):
    a, b = _cases(np.random.default_rng(n), n)
    want = oracle_mod.mul(a, b)
    for i in range(2):
        got = ntt.mul_single_prime(list(map(int, a[i])), list(map(int, b[i])))
        assert got == list(map(int, want[i]))


@pytest.mark.parametrize("na,nb", [(1, 1), (5, 3), (64, 64), (128, 17)])
def test_two_prime_32bit_digits_exact(oracle_mod, na, nb):
    rng = np.random.default_rng(na * 100 + nb)
    a, b = pins.rand_batch(rng, 2, na), pins.rand_batch(rng, 2, nb)
    a[1] = 0xFFFFFFFF
    b[1] = 0xFFFFFFFF
    want = oracle_mod.mul(a, b)
    for i in range(2):
        assert ntt.mul_two_prime(list(map(int, a[i])), list(map(int, b[i]))) == list(map(int, want[i]))


def test_garner_against_small_crt():
    p1, p2 = 97, 193
    for c in range(0, p1 * p2, 37):
        assert ntt.garner(c % p1, c % p2, p1, p2) == c


def test_bounds_at_the_top_of_the_range():
    # 256K-bit operands: 16384 16-bit digits, or 8192 32-bit digits, per side.
    assert ntt.coefficient_bound(16384, 16384, 16) < ntt.PRIME_FIELD_64.p
    assert ntt.coefficient_bound(8192, 8192, 32) < ntt.PRIME_FIELD_64.p * ntt.PRIME_FIELD_CRT2.p
    assert ntt.transform_length(16384, 16384) == 1 << 15
    assert ntt.transform_length(8192, 8192) == 1 << 14


def test_printed_digit_sizes_are_not_exact(oracle_mod):
    """Reading of Section 4.1: PrimeField32 with 15-bit digits admits only 3
    terms per coefficient and PrimeField64 with 31-bit digits admits none, so
    all-ones operands come out wrong; the readings above fix the digit sizes."""
    assert ntt.coefficient_bound(3, 3, 15) < ntt.PRIME_FIELD_32.p < ntt.coefficient_bound(4, 4, 15)
    assert ntt.coefficient_bound(1, 1, 31) > ntt.PRIME_FIELD_64.p
    ones = [0xFFFFFFFF] * 4
    want = list(map(int, oracle_mod.mul(np.array([ones], np.uint32), np.array([ones], np.uint32))[0]))
    assert ntt.mul_single_prime(ones, ones, ntt.PRIME_FIELD_32, d=15) != want
    assert ntt.mul_single_prime(ones, ones, ntt.PRIME_FIELD_64, d=31) != want
    assert ntt.mul_single_prime(ones, ones, ntt.PRIME_FIELD_64, d=16) == want


def test_short_transform_wraps_around():
    """Reading of the padding: a transform shorter than da + db digits wraps the
    top coefficients onto the bottom ones."""
    f = ntt.PRIME_FIELD_64
    xd = [0xFFFF] * 8
    full = ntt.convolve_mod(xd, xd, f)
    assert len(full) == 16
    w = f.root(8)
    short = ntt.intt([u * u % f.p for u in ntt.ntt(xd, w, f.p)], w, f.p)
    assert short == [(full[i] + full[i + 8]) % f.p for i in range(8)]
    assert short != full[:8]


@pytest.mark.parametrize("na,nb", [(1, 1), (2, 7), (33, 31), (64, 64), (100, 3)])
def test_three_prime_32bit_digits_exact(oracle_mod, na, nb):
    rng = np.random.default_rng(na * 1000 + nb + 7)
    a, b = pins.rand_batch(rng, 3, na), pins.rand_batch(rng, 3, nb)
    a[1] = 0xFFFFFFFF
    b[1] = 0xFFFFFFFF
    b[2] = 0
    want = oracle_mod.mul(a, b)
    for i in range(3):
        got = ntt.mul_three_prime(list(map(int, a[i])), list(map(int, b[i])))
        assert got == list(map(int, want[i]))
        x, y = pins.to_int(a[i]), pins.to_int(b[i])
        assert pins.to_int(np.array(got, dtype=np.uint64).astype(np.uint32)) == x * y


def test_garner3_against_brute_force_crt():
    """garner3 returns the unique residue below p0 p1 p2 (checked by search on
    small primes, and on random values for the three 32-bit primes)."""
    small = [5, 7, 11]
    for c in range(5 * 7 * 11):
        assert ntt.garner3([c % q for q in small], small) == c
    ps = [f.p for f in ntt.PRIME_FIELDS_3X32]
    rng = np.random.default_rng(21)
    top = ps[0] * ps[1] * ps[2]
    for _ in range(200):
        c = int(rng.integers(0, 1 << 62)) * int(rng.integers(1, 1 << 26)) % top
        assert ntt.garner3([c % q for q in ps], ps) == c


def test_three_prime_bounds():
    """Three primes below 2^30 (so 4p < 2^32 for lazy 32-bit Montgomery
    arithmetic), 2-adicity covering the longest transform, and a product
    above every coefficient at the top of the range."""
    fs = ntt.PRIME_FIELDS_3X32
    assert len({f.p for f in fs}) == 3
    assert all(f.p < 1 << 30 and f.n >= 15 for f in fs)
    assert ntt.coefficient_bound(8192, 8192, 32) < fs[0].p * fs[1].p * fs[2].p
    # one prime alone is exceeded already by a few all-ones digits
    assert ntt.coefficient_bound(1, 1, 32) > fs[2].p
