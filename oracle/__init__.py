"""CPU oracle for batched midsize integer addition and multiplication.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The product
library never imports, links or calls it, and it shares no code with the CUDA
path: the seeded input generators live in their own module and carry none of
the method's arithmetic.

Contents
--------
``oracle.c`` (built to ``liboracle.so`` by :func:`build`)
    Plain schoolbook addition and multiplication on 64-bit words with 128-bit
    intermediates (Section 2's sequential add-with-carry; Section 3, Eq. (1)).
    Batched with POSIX threads.  This is the parity reference for every GPU
    entry point: all three multiplication variants must equal the same product.
``carry.py``
    The paper's carry-propagation operators and its three-step (map, exclusive
    scan, map) addition, Section 2, on small Python-int cases.
``ntt.py``
    The paper's prime-field construction and a radix-2 number-theoretic
    transform over Python ints (Section 4), used to pin the readings of the
    prime fields, digit sizes and transform lengths.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB_PATH = _HERE / "liboracle.so"


def compile_library(src: Path, out: Path, extra_flags=()) -> Path:
    """Compile a copy of the oracle source into a shared library."""
    tmp = out.with_name(out.name + f".tmp{os.getpid()}")
    cc = os.environ.get("CC", "gcc")
    subprocess.run([cc, "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", *extra_flags,
                    str(src), "-o", str(tmp)], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> Path:
    """Compile ``oracle.c`` into ``liboracle.so`` with the host C compiler."""
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        compile_library(_SRC, _LIB_PATH)
    return _LIB_PATH


def default_threads() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


def _as_batch(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint32)
    if x.ndim == 1:
        x = x[None, :]
    if x.ndim != 2 or x.shape[1] == 0:
        raise ValueError("operands are (batch, limbs) arrays with limbs >= 1")
    return x


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class OracleLib:
    """The oracle's entry points from one compiled copy of ``oracle.c``."""

    def __init__(self, path: Path):
        lib = ctypes.CDLL(str(path))
        u32p = ctypes.POINTER(ctypes.c_uint32)
        for name in ("oracle_add", "oracle_mul"):
            fn = getattr(lib, name)
            fn.argtypes = [u32p, u32p, u32p, ctypes.c_uint32, ctypes.c_uint32,
                           ctypes.c_uint64, ctypes.c_int]
            fn.restype = ctypes.c_int
        lib.oracle_sub.argtypes = [u32p, u32p, u32p, u32p, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]
        lib.oracle_sub.restype = ctypes.c_int
        lib.oracle_mod_u64.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64]
        lib.oracle_mod_u64.restype = ctypes.c_uint64
        self._lib = lib

    def add(self, a: np.ndarray, b: np.ndarray, threads: int | None = None) -> np.ndarray:
        """c = a + b per instance, max(na, nb) + 1 limbs (Section 2)."""
        a, b = _as_batch(a), _as_batch(b)
        if a.shape[0] != b.shape[0]:
            raise ValueError("batch sizes differ")
        c = np.empty((a.shape[0], max(a.shape[1], b.shape[1]) + 1), np.uint32)
        rc = self._lib.oracle_add(_ptr(a), _ptr(b), _ptr(c), a.shape[1], b.shape[1],
                                  a.shape[0], threads or default_threads())
        if rc != 0:
            raise RuntimeError(f"oracle_add failed ({rc})")
        return c

    def sub(self, a: np.ndarray, b: np.ndarray, threads: int | None = None):
        """(a - b mod 2^(32 na), borrow) per instance; requires nb <= na."""
        a, b = _as_batch(a), _as_batch(b)
        c = np.empty_like(a)
        borrow = np.empty(a.shape[0], np.uint32)
        rc = self._lib.oracle_sub(_ptr(a), _ptr(b), _ptr(c), _ptr(borrow), a.shape[1],
                                  b.shape[1], a.shape[0], threads or default_threads())
        if rc != 0:
            raise RuntimeError(f"oracle_sub failed ({rc})")
        return c, borrow

    def mul(self, a: np.ndarray, b: np.ndarray, threads: int | None = None) -> np.ndarray:
        """c = a * b per instance, na + nb limbs (Section 3, Eq. (1))."""
        a, b = _as_batch(a), _as_batch(b)
        if a.shape[0] != b.shape[0]:
            raise ValueError("batch sizes differ")
        c = np.empty((a.shape[0], a.shape[1] + b.shape[1]), np.uint32)
        rc = self._lib.oracle_mul(_ptr(a), _ptr(b), _ptr(c), a.shape[1], b.shape[1],
                                  a.shape[0], threads or default_threads())
        if rc != 0:
            raise RuntimeError(f"oracle_mul failed ({rc})")
        return c

    def mod_u64(self, a: np.ndarray, q: int) -> int:
        """a mod q for one integer given as u32 limbs, 0 < q < 2^63."""
        a = np.ascontiguousarray(a, dtype=np.uint32).ravel()
        return int(self._lib.oracle_mod_u64(_ptr(a), a.size, q))


_default: OracleLib | None = None


def _get() -> OracleLib:
    global _default
    if _default is None:
        _default = OracleLib(build())
    return _default


def add(a, b, threads=None):
    return _get().add(a, b, threads)


def sub(a, b, threads=None):
    return _get().sub(a, b, threads)


def mul(a, b, threads=None):
    return _get().mul(a, b, threads)


def mod_u64(a, q):
    return _get().mod_u64(a, q)
