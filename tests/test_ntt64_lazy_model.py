"""CPU model of the 64-bit transform kernels' field arithmetic: Shoup twiddle
products, Harvey's lazy butterflies with the one-word reduction, the
Montgomery pointwise product and the final scale, run as whole transforms.

It checks the formulation the kernels implement, not the oracle: every
intermediate must stay inside 64 bits (no wrap, no negative difference),
the forward values below 2P and the inverse values below 4P + 2^32 at every
stage, and the transform product must equal the cyclic convolution of the
digits, computed exactly with Python integers (Kronecker substitution).
Planted slips (a subtraction constant that is not a multiple of P, the
one-word reduction in the forward butterflies, the twiddle-1 inverse
butterfly without its exact reduction, the reduction threshold one word too
low) must make a check fail.
"""
import random

import pytest

M64 = (1 << 64) - 1
PRIMES = {"p1": (29 * 2**57 + 1, 21, 57), "p2": (27 * 2**56 + 1, pow(5, 27, 27 * 2**56 + 1), 56)}


class Field:
    """The kernels' Field64<P>, every step checked for 64-bit range."""

    def __init__(self, p, k_extra=0, h_delta=0, lazy_forward=False, lazy_twiddle1=False):
        self.p, self.two_p = p, 2 * p
        self.ph = p >> 32
        self.h = (2 * p >> 32) + h_delta
        self.k = 2 * p + k_extra          # constant added before a subtraction
        self.lazy_forward = lazy_forward
        self.lazy_twiddle1 = lazy_twiddle1

    @staticmethod
    def _w(x):
        assert 0 <= x <= M64, "64-bit range left"
        return x

    def rexact(self, r):
        t = (r - self.two_p) & M64
        return t if t < r else r

    def red(self, r):
        return self._w(r - self.two_p) if (r >> 32) > self.h else r

    def red2(self, r):
        return self.rexact(self.red(r))

    def add(self, a, b):
        s = self._w(a + b)
        return self.red(s) if self.lazy_forward else self.rexact(s)

    def sub(self, a, b):
        s = self._w(self._w(a + self.k) - b)
        return self.red(s) if self.lazy_forward else self.rexact(s)

    def shoup_pair(self, w):
        w %= self.p
        return w, (w << 64) // self.p

    def shoup(self, x, pair):
        w, wq = pair
        q = (x * wq) >> 64
        qp = (q + (((q & 0xFFFFFFFF) * self.ph) << 32)) & M64
        r = ((x * w) & M64) - qp
        r &= M64
        assert r < self.two_p and (r - x * w) % self.p == 0
        return r

    def mont(self, a, b):
        """The kernels' Montgomery product, word by word."""
        assert a < 2**63 and b < 2**63
        m32 = 0xFFFFFFFF
        a0, a1, b0, b1 = a & m32, a >> 32, b & m32, b >> 32
        p00 = a0 * b0
        t = self._w(a0 * b1 + (p00 >> 32))
        t = self._w(t + a1 * b0)
        hi = self._w(a1 * b1 + (t >> 32))
        x0, x1 = p00 & m32, t & m32
        m0 = (-x0) & m32
        m1 = (x0 * self.ph - x1 - (x0 != 0)) & m32
        sm = self._w(m0 * self.ph + m1)
        h = self._w(m1 * self.ph + (sm >> 32))
        r = self._w(hi + h + ((x0 | x1) != 0))
        assert r < self.two_p and (r * 2**64 - a * b) % self.p == 0
        return r

    def dif(self, u, v, w):
        return self.add(u, v), self.shoup(self._w(self._w(u + self.k) - v), w)

    def dif1(self, u, v):
        return self.add(u, v), self.sub(u, v)

    def dit(self, u, v, w):
        x, t = self.red(u), self.shoup(v, w)
        return self._w(x + t), self._w(self._w(x + self.two_p) - t)

    def dit1(self, u, v):
        x = self.red(u)
        t = self.red(v) if self.lazy_twiddle1 else self.red2(v)
        return self._w(x + t), self._w(self._w(x + self.two_p) - t)


def transform_product(f, g, n_log, x, y, one_as_dif1=True):
    """Digits x, y (length L = 2^n_log) -> cyclic convolution mod p, through
    the kernels' sequence: forward DIF (natural in, bit-reversed out),
    Montgomery pointwise, inverse DIT (bit-reversed in, natural out), scale by
    N^-1 R with Shoup, canonical."""
    p = f.p
    L = 1 << n_log
    w = pow(g[0], (1 << g[1]) // L, p)
    wi = pow(w, -1, p)
    A, B = list(x), list(y)
    fwd_bound, inv_bound = 2 * p, 4 * p + 2**32
    h = L // 2
    while h >= 1:                       # DIF stages, half-sizes L/2 .. 1
        wh = pow(w, L // (2 * h), p)
        for buf in (A, B):
            for blk in range(0, L, 2 * h):
                for j in range(h):
                    u, v = buf[blk + j], buf[blk + j + h]
                    if j == 0 and one_as_dif1:
                        buf[blk + j], buf[blk + j + h] = f.dif1(u, v)
                    else:
                        buf[blk + j], buf[blk + j + h] = f.dif(u, v, f.shoup_pair(pow(wh, j, p)))
            assert max(buf) < fwd_bound
        h //= 2
    C = [f.mont(a, b) for a, b in zip(A, B)]
    h = 1
    while h < L:                        # DIT stages, half-sizes 1 .. L/2
        wh = pow(wi, L // (2 * h), p)
        for blk in range(0, L, 2 * h):
            for j in range(h):
                u, v = C[blk + j], C[blk + j + h]
                if j == 0 and one_as_dif1:
                    C[blk + j], C[blk + j + h] = f.dit1(u, v)
                else:
                    C[blk + j], C[blk + j + h] = f.dit(u, v, f.shoup_pair(pow(wh, j, p)))
        assert max(C) < inv_bound
        h *= 2
    scale = f.shoup_pair(pow(L, -1, p) * pow(2, 64, p))
    out = []
    for c in C:
        r = f.shoup(c, scale)
        out.append(r - p if r >= p else r)
    return out


def convolution(x, y):
    """Cyclic convolution of two digit lists by one Python integer product
    (128-bit slots: every coefficient is below L 2^64 < 2^128)."""
    L = len(x)
    X = sum(d << (128 * i) for i, d in enumerate(x))
    Y = sum(d << (128 * i) for i, d in enumerate(y))
    Z = X * Y
    lin = [(Z >> (128 * i)) & ((1 << 128) - 1) for i in range(2 * L)]
    return [lin[i] + lin[i + L] for i in range(L)]


def digits(L, rng, kind, bits=16):
    half = L // 2          # the upper half is zero padding, as in the kernels
    if kind == "max":
        v = [(1 << bits) - 1] * half
    else:
        v = [rng.randrange(1 << bits) for _ in range(half)]
    return v + [0] * (L - half)


@pytest.mark.parametrize("prime", sorted(PRIMES))
@pytest.mark.parametrize("n_log,kind,bits", [(4, "max", 16), (7, "rand", 32), (10, "max", 32),
                                             (13, "max", 16), (13, "rand", 16)])
def test_lazy_transform_product_is_exact(prime, n_log, kind, bits):
    p, g, m = PRIMES[prime]
    if prime == "p2" and bits == 16:
        bits = 32
    f = Field(p)
    rng = random.Random(n_log * 7 + bits)
    L = 1 << n_log
    x, y = digits(L, rng, kind, bits), digits(L, rng, kind, bits)
    got = transform_product(f, (g, m), n_log, x, y, one_as_dif1=(n_log % 2 == 0))
    want = [c % p for c in convolution(x, y)]
    assert got == want


def corner_checks(f):
    """Each butterfly at the corners of its declared input range: outputs
    inside the ranges the next stage assumes, and correct mod P."""
    p = f.p
    fwd = [0, 1, p - 1, p, 2 * p - 2, 2 * p - 1]
    inv = fwd + [2 * p, 3 * p, 4 * p - 1, 4 * p + 2**32 - 1]
    w = f.shoup_pair(pow(3, 12345, p))
    for u in fwd:
        for v in fwd:
            for out, want in ((f.dif(u, v, w), ((u + v) % p, (u - v) * w[0] % p)),
                              (f.dif1(u, v), ((u + v) % p, (u - v) % p))):
                assert all(o < 2 * p for o in out)
                assert (out[0] % p, out[1] % p) == want
    for u in inv:
        for v in inv:
            for out, t in ((f.dit(u, v, w), v * w[0]), (f.dit1(u, v), v)):
                assert all(o < 4 * p + 2**32 for o in out)
                assert (out[0] % p, out[1] % p) == ((u + t) % p, (u - t) % p)


def test_butterfly_corners():
    for p, _, _ in PRIMES.values():
        corner_checks(Field(p))


@pytest.mark.parametrize("slip", ["constant", "lazy_forward", "lazy_twiddle1", "threshold"])
def test_planted_slips_fail(slip):
    p, g, m = PRIMES["p1"]
    kw = {"constant": dict(k_extra=1 << 40), "lazy_forward": dict(lazy_forward=True),
          "lazy_twiddle1": dict(lazy_twiddle1=True), "threshold": dict(h_delta=-1)}[slip]
    f = Field(p, **kw)
    rng = random.Random(3)
    x, y = digits(1 << 10, rng, "max", 32), digits(1 << 10, rng, "max", 32)
    with pytest.raises(AssertionError):
        corner_checks(f)
        got = transform_product(f, (g, m), 10, x, y)
        assert got == [c % p for c in convolution(x, y)]
