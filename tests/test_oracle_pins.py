"""Pins of the CPU oracle (no GPU): each check compares the oracle with a fact
that does not come from the oracle itself; see ``pins.py``."""
import numpy as np
import pytest

import pins


def is_probable_prime(n: int) -> bool:
    if n < 2:
        return False
    small = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:               # deterministic for n < 3.3e24
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(oracle_mod, check):
    check(oracle_mod)


def test_residue_primes_are_prime():
    assert all(is_probable_prime(q) for q in pins.RESIDUE_PRIMES)


def test_truncated_product_is_low_limbs(oracle_mod):
    """Section 2/3 keep results the input length (mod 2^(32 M)); that is the
    low M limbs of the full-width result."""
    rng = np.random.default_rng(11)
    a, b = pins.rand_batch(rng, 5, 64), pins.rand_batch(rng, 5, 64)
    full = oracle_mod.mul(a, b)
    for i in range(5):
        want = (pins.to_int(a[i]) * pins.to_int(b[i])) % (1 << (32 * 64))
        assert pins.to_int(full[i, :64]) == want


def test_empty_batch_and_bad_sizes(oracle_mod):
    z = np.zeros((0, 4), np.uint32)
    assert oracle_mod.mul(z, z).shape == (0, 8)
    with pytest.raises(ValueError):
        oracle_mod.add(np.zeros((1, 0), np.uint32), np.zeros((1, 0), np.uint32))


def test_large_worst_case(oracle_mod):
    """Full 256K-bit size: (2^N - 1)^2 and a random pair against Python ints."""
    n = 8192
    ones = np.full((1, n), 0xFFFFFFFF, np.uint32)
    got = oracle_mod.mul(ones, ones)[0]
    assert pins.to_int(got) == ((1 << (32 * n)) - 1) ** 2
    rng = np.random.default_rng(3)
    a, b = pins.rand_batch(rng, 1, n), pins.rand_batch(rng, 1, n)
    assert pins.to_int(oracle_mod.mul(a, b)[0]) == pins.to_int(a[0]) * pins.to_int(b[0])
