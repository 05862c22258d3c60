"""The split of a long transform into S = 2 or 4 shorter ones (Section 4's
transform, longer than one CTA's shared memory holds), as the transform
kernels run it, checked on the CPU with Python integers over the two 64-bit
primes.

With N = S L and w = w_N, the spectrum X[S k + s] of x (length N) is the
length-L transform of y_s[j] = w^(j s) sum_r x[j + r L] w_S^(r s), and the
inverse recombines c[j + r L] = sum_s w_S^(-r s) (N^-1 w^(-j s) z_s[j]) from
the L-point inverse transforms z_s of the S pointwise products.  The kernels
evaluate both inner sums as radix-2/4 butterflies: w_2 = w_4^2 = -1, so for
S = 4 the only product is by w_4 (times x1 - x3), and sub-problem 0 takes no
w^(j s) factor.  Here those butterflies are written out as the kernels form
them; each L-point transform is its O(L^2) definition; the result must be the
direct cyclic convolution.  Planted mistakes in the butterflies fail."""
import random

import pytest

from oracle import ntt as ontt

FIELDS = [ontt.PRIME_FIELD_64, ontt.PRIME_FIELD_CRT2]


def _dft(x, omega, p):
    n = len(x)
    return [sum(x[j] * pow(omega, j * k, p) for j in range(n)) % p for k in range(n)]


def fold(x, s, S, w, w4, p):
    """Sub-problem s of the forward split: the radix-S butterfly over
    x[j + r L], then w^(j s) (none for s = 0)."""
    L = len(x) // S
    y = []
    for j in range(L):
        x0, x1 = x[j], x[j + L]
        if S == 2:
            acc = (x0 + x1) if s == 0 else (x0 - x1)
        else:
            x2, x3 = x[j + 2 * L], x[j + 3 * L]
            if s == 0:
                acc = (x0 + x2) + (x1 + x3)
            elif s == 2:
                acc = (x0 + x2) - (x1 + x3)
            else:
                o, q = x0 - x2, (x1 - x3) * w4
                acc = o + q if s == 1 else o - q
        if s:
            acc *= pow(w, j * s, p)
        y.append(acc % p)
    return y


def combine(z, S, w, w4i, p):
    """The last inverse radix-S stage: u_s = N^-1 w^(-j s) z_s[j], then the
    radix-S butterfly with the single product by w_4^-1."""
    L = len(z[0])
    N = S * L
    ninv, wi = pow(N, p - 2, p), pow(w, p - 2, p)
    c = [0] * N
    for j in range(L):
        u = [z[s][j] * ninv * pow(wi, j * s, p) % p for s in range(S)]
        if S == 2:
            c[j], c[j + L] = u[0] + u[1], u[0] - u[1]
        else:
            e0, e1 = u[0] + u[2], u[1] + u[3]
            o0, o1 = u[0] - u[2], (u[1] - u[3]) * w4i
            c[j], c[j + L], c[j + 2 * L], c[j + 3 * L] = e0 + e1, o0 + o1, e0 - e1, o0 - o1
    return [v % p for v in c]


def split_convolution(x, y, S, field, fold_fn=fold, combine_fn=combine):
    p, N = field.p, len(x)
    L = N // S
    w = field.root(N)
    wL, w4 = pow(w, S, p), pow(w, N // 4, p)
    w4i = pow(w4, p - 2, p)
    z = []
    for s in range(S):
        X = _dft(fold_fn(x, s, S, w, w4, p), wL, p)
        Y = _dft(fold_fn(y, s, S, w, w4, p), wL, p)
        P = [a * b % p for a, b in zip(X, Y)]
        z.append(_dft(P, pow(wL, p - 2, p), p))     # unscaled inverse
    return combine_fn(z, S, w, w4i, p)


def _inputs(rng, N, bits):
    half = N // 2                                   # zero top half: no wrap-around
    x = [rng.randrange(1 << bits) for _ in range(half)] + [0] * half
    y = [rng.randrange(1 << bits) for _ in range(half)] + [0] * half
    return x, y


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
@pytest.mark.parametrize("S", [2, 4])
@pytest.mark.parametrize("N", [8, 32, 64])
def test_split_equals_cyclic_convolution(field, S, N):
    rng = random.Random(1000 * N + 10 * S + field.k)
    for bits in (16, 32):
        x, y = _inputs(rng, N, bits)
        assert split_convolution(x, y, S, field) == ontt.cyclic_convolution(x, y, field.p)


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_split_all_ones_digits(field):
    """Every digit at its maximum: the largest coefficients, still exact."""
    N = 64
    x = [(1 << 16) - 1] * (N // 2) + [0] * (N // 2)
    for S in (2, 4):
        assert split_convolution(x, x, S, field) == ontt.cyclic_convolution(x, x, field.p)


@pytest.mark.parametrize("field", FIELDS, ids=lambda f: f.name)
def test_butterfly_identities(field):
    """The identities the butterflies rest on: w_2 = w_4^2 = -1 and w^0 = 1."""
    p = field.p
    w4 = field.root(4)
    assert pow(w4, 2, p) == p - 1 and field.root(2) == p - 1
    assert pow(w4, 4, p) == 1 and w4 not in (1, p - 1)


def _swap_r1_r3(z, S, w, w4i, p):
    c = combine(z, S, w, w4i, p)
    L = len(z[0])
    if S == 4:
        c[L:2 * L], c[3 * L:4 * L] = c[3 * L:4 * L], c[L:2 * L]
    return c


def _w4_for_w4inv(z, S, w, w4i, p):
    return combine(z, S, w, pow(w4i, p - 2, p), p)


def _fold_s2_as_s0(x, s, S, w, w4, p):
    return fold(x, 0 if s == 2 else s, S, w, w4, p)


def _fold_no_twiddle(x, s, S, w, w4, p):
    return fold(x, s, S, 1, w4, p)


@pytest.mark.parametrize("mistake", ["swap_r1_r3", "w4_for_w4inv", "fold_s2_as_s0", "fold_no_twiddle"])
def test_planted_mistakes_are_caught(mistake):
    field, S, N = ontt.PRIME_FIELD_64, 4, 32
    x, y = _inputs(random.Random(7), N, 16)
    kw = {"swap_r1_r3": {"combine_fn": _swap_r1_r3}, "w4_for_w4inv": {"combine_fn": _w4_for_w4inv},
          "fold_s2_as_s0": {"fold_fn": _fold_s2_as_s0}, "fold_no_twiddle": {"fold_fn": _fold_no_twiddle}}[mistake]
    assert split_convolution(x, y, S, field, **kw) != ontt.cyclic_convolution(x, y, field.p)
