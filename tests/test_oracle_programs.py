"""Pins of the same-length product and of Section 6's fused programs in the
oracle (no GPU): CPython big integers reduced modulo 2^(32 n), closed forms,
and planted mistakes in copies of ``oracle/programs.py`` that the pins catch."""
from pathlib import Path

import numpy as np
import pytest

import oracle
from oracle import programs
from pins import from_int, rand_batch, to_int

SRC = Path(programs.__file__).read_text()


def _int_programs(x: int, y: int, n: int):
    m = 1 << (32 * n)
    seq = [x, y]
    for _ in range(6):
        seq.append((seq[-1] + seq[-2]) % m)
    return {
        "mul_low": x * y % m,
        "add6": seq[-1],
        "poly": ((x * x + y) * (y * y + y) + x * y) % m,
    }


def _edge_rows(n):
    ones = (1 << (32 * n)) - 1
    return [(ones, ones), (ones, 1), (0, ones), (1, 0), (ones, 0), (1 << (32 * n - 1), 3)]


def check_programs(mod, seed=3):
    rng = np.random.default_rng(seed)
    for n in [1, 2, 3, 8, 33, 64, 129]:
        a, b = rand_batch(rng, 5, n), rand_batch(rng, 5, n)
        rows = [(to_int(a[i]), to_int(b[i])) for i in range(5)] + _edge_rows(n)
        a = np.stack([from_int(x, n) for x, _ in rows])
        b = np.stack([from_int(y, n) for _, y in rows])
        got = {name: getattr(mod, name)(a, b) for name in ("mul_low", "add6", "poly")}
        for i, (x, y) in enumerate(rows):
            want = _int_programs(x, y, n)
            for name, g in got.items():
                assert g.shape == (len(rows), n), (name, g.shape)
                assert to_int(g[i]) == want[name], (name, n, i)


def test_programs_match_python_ints():
    check_programs(programs)


def test_add6_closed_form():
    """x_7 of the chain is 8a + 13b (Fibonacci coefficients F_6, F_7)."""
    rng = np.random.default_rng(11)
    for n in [1, 4, 50]:
        a, b = rand_batch(rng, 4, n), rand_batch(rng, 4, n)
        got = programs.add6(a, b)
        m = 1 << (32 * n)
        for i in range(4):
            assert to_int(got[i]) == (8 * to_int(a[i]) + 13 * to_int(b[i])) % m


def test_poly_at_minus_one():
    """a = 2^(32n) - 1 = -1: (1 + b)(b^2 + b) - b = b^3 + 2 b^2 (mod 2^(32n))."""
    rng = np.random.default_rng(12)
    for n in [1, 5, 40]:
        b = rand_batch(rng, 3, n)
        a = np.full_like(b, 0xFFFFFFFF)
        got = programs.poly(a, b)
        m = 1 << (32 * n)
        for i in range(3):
            y = to_int(b[i])
            assert to_int(got[i]) == (y ** 3 + 2 * y * y) % m


def test_mul_low_is_low_half_of_full_product():
    rng = np.random.default_rng(13)
    a, b = rand_batch(rng, 7, 70), rand_batch(rng, 7, 70)
    assert np.array_equal(programs.mul_low(a, b), oracle.mul(a, b)[:, :70])


MUTANTS = [
    ("add6_five_steps", "for _ in range(6):", "for _ in range(5):"),
    ("add6_keeps_operand", "prev, cur = cur, add_low(cur, prev, threads)",
     "prev, cur = prev, add_low(cur, prev, threads)"),
    ("poly_drops_b_term", "t2 = add_low(mul_low(b, b, threads), b, threads)",
     "t2 = mul_low(b, b, threads)"),
    ("poly_squares_a_twice", "t4 = mul_low(a, b, threads)", "t4 = mul_low(a, a, threads)"),
    ("low_keeps_high_limb", "return np.ascontiguousarray(x[:, :n])",
     "return np.ascontiguousarray(x[:, 1:n + 1])"),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_program_mutant_is_caught(name, orig, bad):
    assert SRC.count(orig) == 1, "mutation anchor must be unique"
    ns = {"__name__": f"oracle._mutant_{name}", "__package__": "oracle"}
    exec(compile(SRC.replace(orig, bad), f"<{name}>", "exec"), ns)

    class Mutant:
        mul_low = staticmethod(ns["mul_low"])
        add6 = staticmethod(ns["add6"])
        poly = staticmethod(ns["poly"])

    with pytest.raises(AssertionError):
        check_programs(Mutant)
