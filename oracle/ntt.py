"""Prime fields and the number-theoretic transform of Section 4, on Python ints.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow; small cases.

Section 4.1 builds fields Z_p for primes of the form ``p = k * 2^n + 1``.  By
Fermat's little theorem every ``a`` satisfies ``a^(k 2^n) = 1 (mod p)``, so
``g = a^k`` satisfies ``g^(2^n) = 1``; the first ``a`` whose ``g`` has order
exactly ``2^n`` gives a primitive ``2^n``-th root of unity, and for a power of
two ``M <= 2^n`` the element ``omega = g^(2^n / M)`` is a primitive ``M``-th
root.  The paper prints two such fields (PrimeField32 and PrimeField64 below).

Section 4.2 multiplies integers by transforming digit vectors, multiplying the
spectra pointwise and transforming back with ``omega^-1`` and a final ``M^-1``
scale; the coefficients are then carried back into machine words.

Readings taken here (the paper is silent or inexact on these points):

* Transform length.  A cyclic convolution of length ``M`` wraps around unless
  ``M`` is at least the number of product digits, so ``M`` is the next power of
  two >= digits(a) + digits(b), and the digits above the inputs are zero.
* Digit size.  Every convolution coefficient must stay below ``p`` for the
  result to be exact: ``min(da, db) * (2^d - 1)^2 < p``.  The paper's
  PrimeField32 with 15-bit digits admits at most 3 terms and PrimeField64 with
  31-bit digits admits none, so neither is exact at midsize lengths.  The
  single-prime form used here takes PrimeField64 with 16-bit digits (bound
  < 2^46 for the 256K-bit range); the two-prime form takes 32-bit digits over
  PrimeField64 and a second good prime, ``27 * 2^56 + 1`` (root 5^27 of order
  2^56), and recombines by CRT (bound < 2^77 < p1 * p2 ~ 2^122.6).  Any prime
  k * 2^n + 1 with 2^n >= the transform length is equally valid; this one is
  chosen, like p1, with low 32-bit word 1 and below 2^62.
* ``g`` as printed is itself a primitive ``2^n``-th root of unity (verified in
  the tests), and ``omega_M = g^(2^n / M)``.
* Three-prime form (not in the paper; Section 4 uses one field per product).
  32-bit digits over three good primes below 2^30 -- 7 * 2^26 + 1,
  45 * 2^24 + 1 and 119 * 2^23 + 1 -- recombined by Garner's mixed-radix CRT.
  Their product (~2^88.2) exceeds the coefficient bound N (2^32 - 1)^2 for
  every transform length up to 2^23, and primes below 2^30 are what lets a
  GPU keep field elements in 32-bit words with lazy reductions.  Each root is
  the first hit of Section 4.1's search.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence


@dataclass(frozen=True)
class PrimeField:
    """``p = k * 2^n + 1`` with ``g`` a primitive ``2^n``-th root of unity."""
    name: str
    p: int
    k: int
    n: int
    g: int

    def root(self, m: int) -> int:
        """A primitive m-th root of unity for a power of two m <= 2^n."""
        if m <= 0 or m & (m - 1) or m > (1 << self.n):
            raise ValueError("m must be a power of two not above 2^n")
        return pow(self.g, (1 << self.n) // m, self.p)


# Printed in Section 4.1.
PRIME_FIELD_32 = PrimeField("PrimeField32", 3221225473, 3, 30, 13)
PRIME_FIELD_64 = PrimeField("PrimeField64", 4179340454199820289, 29, 57, 21)
# Second CRT prime (a reading, not in the paper): 27 * 2^56 + 1.  a = 5 is the
# first a whose a^27 has order exactly 2^56 (Section 4.1's search).
_P_CRT2 = 27 * (1 << 56) + 1
PRIME_FIELD_CRT2 = PrimeField("CRT2", _P_CRT2, 27, 56, pow(5, 27, _P_CRT2))


def _search_root_field(name: str, k: int, n: int) -> PrimeField:
    p = k * (1 << n) + 1
    return PrimeField(name, p, k, n, search_root(p, k, n))


def search_root(p: int, k: int, n: int, limit: int = 1000) -> int:
    """Section 4.1's search: the first a >= 2 whose a^k has order exactly 2^n."""
    for a in range(2, limit):
        g = pow(a, k, p)
        if pow(g, 1 << (n - 1), p) != 1:     # g^(2^n) = 1 always holds
            return g
    raise ValueError("no root found below the search limit")


def powers(omega: int, m: int, p: int) -> List[int]:
    """[1, omega, omega^2, ..., omega^(m-1)]: an exclusive multiplicative scan."""
    out, acc = [], 1
    for _ in range(m):
        out.append(acc)
        acc = acc * omega % p
    return out


def dft(x: Sequence[int], omega: int, p: int) -> List[int]:
    """The transform by its definition: X_j = sum_i x_i omega^(i j) mod p."""
    m = len(x)
    return [sum(x[i] * pow(omega, i * j, p) for i in range(m)) % p for j in range(m)]


def _bit_reverse(i: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


def ntt(x: Sequence[int], omega: int, p: int) -> List[int]:
    """Radix-2 decimation-in-time transform: bit-reversed reorder, then log2 m
    rounds of butterflies; round with span ``h`` pairs element ``j`` of each
    block of ``2h`` with element ``j + h`` using the twiddle ``omega^(j m/(2h))``.
    Equal to :func:`dft` for the same ``omega``."""
    m = len(x)
    bits = m.bit_length() - 1
    if m == 0 or (1 << bits) != m:
        raise ValueError("length must be a power of two")
    tw = powers(omega, max(m // 2, 1), p)
    y = [x[_bit_reverse(i, bits)] % p for i in range(m)]
    h = 1
    while h < m:
        step = m // (2 * h)
        for start in range(0, m, 2 * h):
            for j in range(h):
                u = y[start + j]
                v = y[start + j + h] * tw[j * step] % p
                y[start + j] = (u + v) % p
                y[start + j + h] = (u - v) % p
        h *= 2
    return y


def intt(y: Sequence[int], omega: int, p: int) -> List[int]:
    """Inverse transform: the forward one with omega^-1, then a scale by m^-1."""
    m = len(y)
    inv_m = pow(m, -1, p)
    return [v * inv_m % p for v in ntt(y, pow(omega, -1, p), p)]


def cyclic_convolution(x: Sequence[int], y: Sequence[int], p: int) -> List[int]:
    """z_k = sum_{i + j = k mod m} x_i y_j mod p, by its definition."""
    m = len(x)
    z = [0] * m
    for i in range(m):
        for j in range(m):
            z[(i + j) % m] = (z[(i + j) % m] + x[i] * y[j]) % p
    return z


# ---- integer multiplication through the transform ------------------------

def limbs_to_int(limbs: Sequence[int], w: int = 32) -> int:
    v = 0
    for limb in reversed(list(limbs)):
        v = (v << w) | int(limb)
    return v


def int_to_limbs(v: int, count: int, w: int = 32) -> List[int]:
    mask = (1 << w) - 1
    out = []
    for _ in range(count):
        out.append(v & mask)
        v >>= w
    if v:
        raise ValueError("value does not fit in the requested limb count")
    return out


def to_digits(limbs: Sequence[int], d: int, w: int = 32) -> List[int]:
    """Split w-bit limbs into d-bit digits, least significant first."""
    v, count = limbs_to_int(limbs, w), (len(limbs) * w + d - 1) // d
    mask = (1 << d) - 1
    return [(v >> (d * i)) & mask for i in range(count)]


def transform_length(da: int, db: int) -> int:
    """Next power of two >= da + db (no cyclic wrap-around)."""
    m = 1
    while m < da + db:
        m *= 2
    return m


def coefficient_bound(da: int, db: int, d: int) -> int:
    """Largest possible convolution coefficient for da- and db-digit inputs."""
    return min(da, db) * ((1 << d) - 1) ** 2


def convolve_mod(xd: Sequence[int], yd: Sequence[int], field: PrimeField) -> List[int]:
    """Cyclic convolution of the zero-padded digit vectors via the transform."""
    m = transform_length(len(xd), len(yd))
    omega = field.root(m)
    xs = list(xd) + [0] * (m - len(xd))
    ys = list(yd) + [0] * (m - len(yd))
    fx, fy = ntt(xs, omega, field.p), ntt(ys, omega, field.p)
    return intt([u * v % field.p for u, v in zip(fx, fy)], omega, field.p)


def mul_single_prime(a: Sequence[int], b: Sequence[int], field: PrimeField = PRIME_FIELD_64,
                     d: int = 16) -> List[int]:
    """a * b (u32 limbs in, len(a)+len(b) limbs out) through one prime field.

    Exact only when :func:`coefficient_bound` is below ``field.p``; otherwise
    the coefficients come back reduced mod p and the product is wrong, which
    the tests use to pin the digit-size reading.
    """
    coeffs = convolve_mod(to_digits(a, d), to_digits(b, d), field)
    value = sum(c << (d * k) for k, c in enumerate(coeffs))
    return int_to_limbs(value % (1 << (32 * (len(a) + len(b)))), len(a) + len(b))


def garner(r1: int, r2: int, p1: int, p2: int) -> int:
    """The unique c < p1 p2 with c = r1 (mod p1) and c = r2 (mod p2)."""
    v = (r2 - r1) * pow(p1, -1, p2) % p2
    return r1 + p1 * v


def mul_two_prime(a: Sequence[int], b: Sequence[int], d: int = 32,
                  f1: PrimeField = PRIME_FIELD_64, f2: PrimeField = PRIME_FIELD_CRT2) -> List[int]:
    """a * b with d-bit digits, two prime fields and Garner recombination."""
    xd, yd = to_digits(a, d), to_digits(b, d)
    c1 = convolve_mod(xd, yd, f1)
    c2 = convolve_mod(xd, yd, f2)
    coeffs = [garner(u, v, f1.p, f2.p) for u, v in zip(c1, c2)]
    value = sum(c << (d * k) for k, c in enumerate(coeffs))
    return int_to_limbs(value % (1 << (32 * (len(a) + len(b)))), len(a) + len(b))


# ---- three 32-bit primes ---------------------------------------------------

PRIME_FIELDS_3X32 = (
    _search_root_field("P32a", 7, 26),     # 469762049
    _search_root_field("P32b", 45, 24),    # 754974721
    _search_root_field("P32c", 119, 23),   # 998244353
)


def garner3(r: Sequence[int], p: Sequence[int]) -> int:
    """The unique c < p0 p1 p2 with c = r_i (mod p_i), by mixed radix:
    c = v0 + v1 p0 + v2 p0 p1 with v0 = r0, v1 = (r1 - v0) / p0 mod p1,
    v2 = ((r2 - v0) / p0 - v1) / p1 mod p2."""
    v0 = r[0]
    v1 = (r[1] - v0) * pow(p[0], -1, p[1]) % p[1]
    v2 = ((r[2] - v0) * pow(p[0], -1, p[2]) - v1) * pow(p[1], -1, p[2]) % p[2]
    return v0 + v1 * p[0] + v2 * p[0] * p[1]


def mul_three_prime(a: Sequence[int], b: Sequence[int], d: int = 32,
                    fields: Sequence[PrimeField] = PRIME_FIELDS_3X32) -> List[int]:
    """a * b with d-bit digits, three prime fields and Garner recombination."""
    xd, yd = to_digits(a, d), to_digits(b, d)
    residues = [convolve_mod(xd, yd, f) for f in fields]
    coeffs = [garner3(rs, [f.p for f in fields]) for rs in zip(*residues)]
    value = sum(c << (d * k) for k, c in enumerate(coeffs))
    return int_to_limbs(value % (1 << (32 * (len(a) + len(b)))), len(a) + len(b))
