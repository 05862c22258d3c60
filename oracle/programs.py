"""Oracle for the same-length product and Section 6's two fused programs.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product
library imports this module.

The paper keeps every result at the operands' length (Section 2), so each step
below is the full oracle result of ``oracle.add`` / ``oracle.mul`` cut back to
n limbs, i.e. arithmetic modulo 2^(32 n).  The programs follow Section 6:

* ``mul_low``: one product, c = a*b mod 2^(32n) (the paper's 1-Mul);
* ``add6``: six additions (6-Add).  The paper names the count but not the
  chain; the reading used here is the dependent chain x_{k+1} = x_k + x_{k-1}
  with x_0 = a, x_1 = b, result x_7, so every addition consumes the previous
  one's result and none can be skipped;
* ``poly``: (a*a + b)*(b*b + b) + a*b (Poly), evaluated in the order the
  expression is written.  The paper counts it as four products and two
  additions; the expression as printed has three additions, which is what is
  computed.

Pins (tests/test_oracle_programs.py): Python big-int arithmetic on small random
and edge inputs, and the closed forms 8a + 13b and a = -1.
"""
from __future__ import annotations

import numpy as np

from . import add as _add
from . import mul as _mul


def _low(x: np.ndarray, n: int) -> np.ndarray:
    """The low n limbs of each row (reduction modulo 2^(32 n))."""
    return np.ascontiguousarray(x[:, :n])


def _check(a: np.ndarray, b: np.ndarray) -> int:
    if a.ndim != 2 or a.shape != b.shape:
        raise ValueError("a and b must be (batch, n) arrays of the same shape")
    return a.shape[1]


def mul_low(a, b, threads=None):
    """a*b mod 2^(32 n) per row."""
    n = _check(a, b)
    return _low(_mul(a, b, threads), n)


def add_low(a, b, threads=None):
    """a + b mod 2^(32 n) per row."""
    n = _check(a, b)
    return _low(_add(a, b, threads), n)


def add6(a, b, threads=None):
    """x_7 of x_{k+1} = x_k + x_{k-1}, x_0 = a, x_1 = b, mod 2^(32 n)."""
    _check(a, b)
    prev, cur = a, b
    for _ in range(6):
        prev, cur = cur, add_low(cur, prev, threads)
    return cur


def poly(a, b, threads=None):
    """(a*a + b)*(b*b + b) + a*b mod 2^(32 n) per row."""
    _check(a, b)
    t1 = add_low(mul_low(a, a, threads), b, threads)
    t2 = add_low(mul_low(b, b, threads), b, threads)
    t3 = mul_low(t1, t2, threads)
    t4 = mul_low(a, b, threads)
    return add_low(t3, t4, threads)
