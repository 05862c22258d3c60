"""Thin ctypes binding over the C ABI of ``include/bn.h``.

Argument marshalling only: every step of every operation runs in the CUDA
library.  There is no CPU fallback; if the library is missing or fails to
load, every entry point raises.  Operands are torch CUDA tensors of dtype
int32 or uint32 (limb bit patterns), shaped (batch, limbs) and contiguous;
results come back as int32 tensors holding u32 bit patterns.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _build

BN_OK, BN_EINVAL, BN_ENOMEM, BN_ECUDA, BN_EUNSUPPORTED, BN_ETIMEOUT = range(6)
(BN_OP_ADD, BN_OP_MUL_QUAD, BN_OP_MUL_NTT64, BN_OP_MUL_NTT_CRT, BN_OP_MUL_AUTO, BN_OP_MUL_NTT3,
 BN_OP_MUL_QUAD_TC) = range(7)
BN_BATCH_AUTOTUNE, BN_BATCH_PLAIN, BN_BATCH_PLAIN_CLASSES = 1, 2, 4
# Layout of struct bn_batch_item (include/bn.h), 40 bytes.
BATCH_ITEM_DTYPE = np.dtype([("op", "<u4"), ("na", "<u4"), ("nb", "<u4"), ("reserved", "<u4"),
                             ("a_offset", "<u8"), ("b_offset", "<u8"), ("c_offset", "<u8")])
BN_ADD_MAX_LIMBS = 16384
BN_MUL_MAX_LIMBS = 8192

_lib = None


class BnError(RuntimeError):
    """A non-OK bn_status, with the library's error text."""

    def __init__(self, status: int, where: str):
        self.status = status
        lib = _lib
        text = lib.bn_status_str(status).decode() if lib else str(status)
        detail = lib.bn_last_error().decode() if lib else ""
        super().__init__(f"{where}: {text}" + (f" ({detail})" if detail else ""))


class bn_batch_info(ctypes.Structure):
    _fields_ = [("classes", ctypes.c_uint32), ("launches", ctypes.c_uint32),
                ("items_add", ctypes.c_uint64), ("items_quad", ctypes.c_uint64),
                ("items_ntt64", ctypes.c_uint64), ("items_crt", ctypes.c_uint64),
                ("tune_ms", ctypes.c_double), ("items_ntt3", ctypes.c_uint64)]


class bn_server_config(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class bn_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("pool_high_water", ctypes.c_uint64),
                ("max_inflight_seen", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


# Layouts of struct bn_request and struct bn_completion (include/bn.h), 40 bytes each.
REQUEST_DTYPE = np.dtype([("op", "<u4"), ("na", "<u4"), ("nb", "<u4"), ("reserved", "<u4"),
                          ("a", "<u8"), ("b", "<u8"), ("arrival_us", "<f8")])
COMPLETION_DTYPE = np.dtype([("ticket", "<u8"), ("c", "<u8"), ("limbs", "<u4"), ("reserved", "<u4"),
                             ("arrival_us", "<f8"), ("done_us", "<f8")])
BN_SERVER_SEQUENTIAL = 1


class bn_tuning(ctypes.Structure):
    _fields_ = [("limbs_per_thread", ctypes.c_uint32), ("cta_threads", ctypes.c_uint32),
                ("variant", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def library_path():
    return _build.library_path()


def load(build_if_missing: bool = False):
    """Load the library (once).  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.library_path()
    if build_if_missing and not _build.is_current():
        _build.build()
    if not path.exists():
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(str(path))
    u32p, vp, u32, u64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    st = ctypes.c_int
    sigs = {
        "bn_plan_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, u32, u32, u64,
                            ctypes.POINTER(bn_tuning)], st),
        "bn_plan_execute": ([vp, u32p, u32p, u32p, vp], st),
        "bn_plan_execute_host": ([vp, u32p, u32p, u32p, vp], st),
        "bn_plan_execute_host_async": ([vp, u32p, u32p, u32p, vp], st),
        "bn_plan_destroy": ([vp], st),
        "bn_plan_out_limbs": ([vp], u32),
        "bn_plan_scratch_bytes": ([vp], ctypes.c_size_t),
        "bn_plan_transform_length": ([vp], u32),
        "bn_add": ([u32p, u32p, u32p, u32, u32, u64, vp], st),
        "bn_mul_quad": ([u32p, u32p, u32p, u32, u32, u64, vp], st),
        "bn_mul_ntt": ([u32p, u32p, u32p, u32, u32, u64, ctypes.c_int, vp], st),
        "bn_mul_ntt3": ([u32p, u32p, u32p, u32, u32, u64, vp], st),
        "bn_mul": ([u32p, u32p, u32p, u32, u32, u64, vp], st),
        "bn_mul_quad_tc": ([u32p, u32p, u32p, u32, u32, u64, vp], st),
        "bn_tc_check": ([], st),
        "bn_tc_wait_selftest": ([u32], st),
        "bn_plan_op": ([vp], ctypes.c_int),
        "bn_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "bn_last_error": ([], ctypes.c_char_p),
        "bn_version": ([], ctypes.c_int),
        "bn_debug_word": ([], ctypes.c_uint32),
        "bn_debug_build": ([], ctypes.c_int),
        "bn_mul_ntt_noalloc": ([u32p, u32p, u32p, u32, u32, u64, ctypes.c_int, vp], st),
        "bn_mul_low": ([u32p, u32p, u32p, u32, u64, vp], st),
        "bn_poly": ([u32p, u32p, u32p, u32, u64, vp], st),
        "bn_add6": ([u32p, u32p, u32p, u32, u64, vp], st),
        "bn_server_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(bn_server_config)], st),
        "bn_server_submit": ([vp, vp, u32, vp], st),
        "bn_server_poll": ([vp, vp, u32, ctypes.POINTER(ctypes.c_uint32)], st),
        "bn_server_release": ([vp, vp, u32], st),
        "bn_server_drain": ([vp, ctypes.c_double], st),
        "bn_server_now_us": ([vp], ctypes.c_double),
        "bn_server_get_stats": ([vp, ctypes.POINTER(bn_server_stats)], st),
        "bn_server_destroy": ([vp], st),
        "bn_batch_create": ([ctypes.POINTER(ctypes.c_void_p), vp, u64, u32], st),
        "bn_batch_execute": ([vp, u32p, u32p, u32p, vp], st),
        "bn_batch_get_info": ([vp, ctypes.POINTER(bn_batch_info)], st),
        "bn_batch_destroy": ([vp], st),
        "bn_probe_int_throughput": ([ctypes.c_int, u32, u32, u32, u32p,
                                     ctypes.POINTER(ctypes.c_uint64), vp], st),
        "bn_probe_mma_throughput": ([u32, u32, u32, u32, u32, u32p, vp], st),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != BN_OK:
        raise BnError(status, where)


def _torch():
    import torch
    return torch


def _operand(x, name):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError(f"{name} must hold 32-bit limbs (int32 or uint32)")
    if x.dim() != 2 or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (batch, limbs) tensor")
    return x


def _stream_handle(stream, device):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _out(out, batch, limbs, like):
    torch = _torch()
    if out is None:
        return torch.empty((batch, limbs), dtype=torch.int32, device=like.device)
    out = _operand(out, "out")
    if tuple(out.shape) != (batch, limbs):
        raise ValueError(f"out must have shape {(batch, limbs)}")
    return out


def _pair(a, b):
    a, b = _operand(a, "a"), _operand(b, "b")
    if a.shape[0] != b.shape[0] or a.device != b.device:
        raise ValueError("a and b need the same batch size and device")
    return a, b


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def bn_add(a, b, out=None, stream=None):
    """c = a + b per row (Section 2); result has max(na, nb) + 1 limbs."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, max(na, nb) + 1, a)
    _check(lib.bn_add(_ptr(a), _ptr(b), _ptr(out), na, nb, batch, _stream_handle(stream, a.device)),
           "bn_add")
    return out


def bn_mul_quad(a, b, out=None, stream=None):
    """c = a * b per row by the classical method (Section 3); na + nb limbs."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    _check(lib.bn_mul_quad(_ptr(a), _ptr(b), _ptr(out), na, nb, batch,
                           _stream_handle(stream, a.device)), "bn_mul_quad")
    return out


def bn_mul_ntt(a, b, crt: bool = False, out=None, stream=None):
    """c = a * b per row through a number-theoretic transform (Section 4)."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    _check(lib.bn_mul_ntt(_ptr(a), _ptr(b), _ptr(out), na, nb, batch, int(bool(crt)),
                          _stream_handle(stream, a.device)), "bn_mul_ntt")
    return out


def bn_mul(a, b, out=None, stream=None):
    """c = a * b per row by the product the cost model finds fastest for the
    sizes (schoolbook or a transform); na + nb limbs."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    _check(lib.bn_mul(_ptr(a), _ptr(b), _ptr(out), na, nb, batch, _stream_handle(stream, a.device)),
           "bn_mul")
    return out


def bn_mul_ntt3(a, b, out=None, stream=None):
    """c = a * b per row through transforms over three 32-bit primes with
    32-bit digits and Garner recombination (Section 4's method); na + nb limbs."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    _check(lib.bn_mul_ntt3(_ptr(a), _ptr(b), _ptr(out), na, nb, batch,
                           _stream_handle(stream, a.device)), "bn_mul_ntt3")
    return out


def bn_mul_quad_tc(a, b, out=None, stream=None):
    """c = a * b per row by the classical method computed on bytes as an exact
    fp16 contraction on the tensor cores (Section 3's column sums); na + nb limbs."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    _check(lib.bn_mul_quad_tc(_ptr(a), _ptr(b), _ptr(out), na, nb, batch,
                              _stream_handle(stream, a.device)), "bn_mul_quad_tc")
    return out


def bn_tc_check():
    """Synchronise the device and raise BnError (BN_ETIMEOUT) if a tensor-core
    kernel gave up waiting for its MMAs since the last check."""
    _check(load().bn_tc_check(), "bn_tc_check")


def bn_tc_wait_selftest(limit_us: int = 20000) -> int:
    """Run the bounded-wait diagnostic; returns the bn_status (BN_ETIMEOUT when
    the waits gave up as designed)."""
    return load().bn_tc_wait_selftest(int(limit_us))


def _same_length(name, a, b, out, stream):
    lib = load()
    a, b = _pair(a, b)
    if a.shape[1] != b.shape[1]:
        raise ValueError(f"{name}: a and b need the same limb count")
    batch, n = a.shape[0], a.shape[1]
    out = _out(out, batch, n, a)
    _check(getattr(lib, name)(_ptr(a), _ptr(b), _ptr(out), n, batch,
                              _stream_handle(stream, a.device)), name)
    return out


def bn_mul_low(a, b, out=None, stream=None):
    """c = a * b mod 2^(32 n) per row: the low half of the classical product,
    n limbs like the operands (Section 3, Fig. 3)."""
    return _same_length("bn_mul_low", a, b, out, stream)


def bn_poly(a, b, out=None, stream=None):
    """c = (a*a + b)*(b*b + b) + a*b mod 2^(32 n) per row, one fused kernel
    (Section 6's polynomial program)."""
    return _same_length("bn_poly", a, b, out, stream)


def bn_add6(a, b, out=None, stream=None):
    """Six dependent additions x_{k+1} = x_k + x_{k-1} from x_0 = a, x_1 = b,
    i.e. c = 8a + 13b mod 2^(32 n) per row, one fused kernel (Section 6)."""
    return _same_length("bn_add6", a, b, out, stream)


def bn_mul_ntt_noalloc(a, b, crt: bool = False, out=None, stream=None):
    """As bn_mul_ntt, but the library allocates nothing: scratch and tables
    live in fixed device arrays shared by all calls (see include/bn.h), for
    callers that cannot call cudaMalloc.  Pass `out` to allocate nothing here
    either; calls that overlap on the GPU race."""
    lib = load()
    a, b = _pair(a, b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    out = _out(out, batch, na + nb, a)
    # The library keys its arrays on the current device: make it a's device.
    with _torch().cuda.device(a.device):
        _check(lib.bn_mul_ntt_noalloc(_ptr(a), _ptr(b), _ptr(out), na, nb, batch, int(bool(crt)),
                                      _stream_handle(stream, a.device)), "bn_mul_ntt_noalloc")
    return out


PROBE_MAD_LO, PROBE_MAD_HI, PROBE_MAD_WIDE, PROBE_MAC_CHAIN = range(4)


def bn_probe_int_throughput(kind: int, blocks: int, threads: int, iters: int, out, stream=None) -> int:
    """Enqueue the integer multiply-add probe; returns multiply-adds per thread."""
    lib = load()
    out = _operand(out, "out") if out.dim() == 2 else out
    ops = ctypes.c_uint64()
    _check(lib.bn_probe_int_throughput(kind, blocks, threads, iters, _ptr(out), ctypes.byref(ops),
                                       _stream_handle(stream, out.device)), "bn_probe_int_throughput")
    return ops.value


def bn_probe_mma_throughput(n: int, chains: int, chain_len: int, iters: int, ctas: int, status,
                            stream=None) -> None:
    """Enqueue the tensor-core chain probe; status: a 1-element int32 device tensor."""
    lib = load()
    _check(lib.bn_probe_mma_throughput(n, chains, chain_len, iters, ctas, _ptr(status),
                                       _stream_handle(stream, status.device)), "bn_probe_mma_throughput")


class Plan:
    """A bn_plan: fixed op, sizes and batch; reusable across calls."""

    def __init__(self, op: int, na: int, nb: int, batch: int,
                 limbs_per_thread: int = 0, cta_threads: int = 0, variant: int = 0):
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        tun = bn_tuning(limbs_per_thread, cta_threads, variant, 0)
        _check(lib.bn_plan_create(ctypes.byref(self._h), op, na, nb, batch, ctypes.byref(tun)),
               "bn_plan_create")
        self.na, self.nb, self.batch = na, nb, batch
        self.op = lib.bn_plan_op(self._h)  # the concrete op (an AUTO plan's choice)
        self.out_limbs = lib.bn_plan_out_limbs(self._h)

    @property
    def scratch_bytes(self) -> int:
        return self._lib.bn_plan_scratch_bytes(self._h)

    @property
    def transform_length(self) -> int:
        return self._lib.bn_plan_transform_length(self._h)

    def execute(self, a, b, out=None, stream=None):
        """Run on device tensors a (batch, na), b (batch, nb)."""
        a, b = _pair(a, b)
        if tuple(a.shape) != (self.batch, self.na) or tuple(b.shape) != (self.batch, self.nb):
            raise ValueError("operand shapes do not match the plan")
        out = _out(out, self.batch, self.out_limbs, a)
        _check(self._lib.bn_plan_execute(self._h, _ptr(a), _ptr(b), _ptr(out),
                                         _stream_handle(stream, a.device)), "bn_plan_execute")
        return out

    def execute_host(self, a: np.ndarray, b: np.ndarray, out: Optional[np.ndarray] = None,
                     stream=None) -> np.ndarray:
        """Run on host arrays (numpy uint32, or pinned torch CPU tensors); the
        library copies in, computes, copies out and synchronises."""
        def host_ptr(x, shape, name):
            if hasattr(x, "data_ptr"):  # torch CPU tensor (possibly pinned)
                if tuple(x.shape) != shape or not x.is_contiguous() or x.element_size() != 4:
                    raise ValueError(f"{name} must be a contiguous 32-bit {shape} tensor")
                return ctypes.c_void_p(x.data_ptr()), x
            arr = np.ascontiguousarray(x, dtype=np.uint32)
            if arr.shape != shape:
                raise ValueError(f"{name} must have shape {shape}")
            return ctypes.c_void_p(arr.ctypes.data), arr
        pa, ka = host_ptr(a, (self.batch, self.na), "a")
        pb, kb = host_ptr(b, (self.batch, self.nb), "b")
        if out is None:
            out = np.empty((self.batch, self.out_limbs), np.uint32)
        pc, kc = host_ptr(out, (self.batch, self.out_limbs), "out")
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(self._lib.bn_plan_execute_host(self._h, pa, pb, pc, ctypes.c_void_p(s.cuda_stream)),
               "bn_plan_execute_host")
        return kc

    def execute_host_async(self, a, b, out, stream=None):
        """Enqueue copy-in, kernel and copy-out on `stream` without waiting
        (bn_plan_execute_host_async).  a, b and out must be contiguous pinned
        torch CPU tensors of 32-bit limbs that the caller keeps alive, a and b
        unchanged, until the stream has passed this call."""
        ptrs = []
        for x, shape, name in ((a, (self.batch, self.na), "a"), (b, (self.batch, self.nb), "b"),
                               (out, (self.batch, self.out_limbs), "out")):
            if not hasattr(x, "data_ptr") or x.is_cuda or not x.is_pinned():
                raise TypeError(f"{name} must be a pinned torch CPU tensor")
            if tuple(x.shape) != shape or not x.is_contiguous() or x.element_size() != 4:
                raise ValueError(f"{name} must be a contiguous 32-bit {shape} tensor")
            ptrs.append(ctypes.c_void_p(x.data_ptr()))
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(self._lib.bn_plan_execute_host_async(self._h, *ptrs, ctypes.c_void_p(s.cuda_stream)),
               "bn_plan_execute_host_async")
        return out

    def close(self):
        if self._h:
            _check(self._lib.bn_plan_destroy(self._h), "bn_plan_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A bn_batch: a fixed list of mixed-size operations over flat arrays.

    ``items`` is a numpy array of BATCH_ITEM_DTYPE (op, na, nb, offsets in
    limbs into the flat a, b, c arrays).  ``execute`` runs them as one CUDA
    graph (or, with BN_BATCH_PLAIN, as one launch per item; with
    BN_BATCH_PLAIN_CLASSES, as one padded plain launch per size class)."""

    def __init__(self, items: np.ndarray, flags: int = 0):
        lib = load()
        self._lib = lib
        items = np.ascontiguousarray(items, dtype=BATCH_ITEM_DTYPE)
        self.items = items
        self._h = ctypes.c_void_p()
        _check(lib.bn_batch_create(ctypes.byref(self._h), ctypes.c_void_p(items.ctypes.data),
                                   items.shape[0], flags), "bn_batch_create")

    @property
    def info(self) -> dict:
        inf = bn_batch_info()
        _check(self._lib.bn_batch_get_info(self._h, ctypes.byref(inf)), "bn_batch_get_info")
        return {k: getattr(inf, k) for k, _ in bn_batch_info._fields_}

    def execute(self, a, b, c, stream=None):
        """Run on flat device tensors (1-D, 32-bit limbs)."""
        for t, name in ((a, "a"), (b, "b"), (c, "c")):
            if not t.is_cuda or t.element_size() != 4 or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous 32-bit CUDA tensor")
        _check(self._lib.bn_batch_execute(self._h, _ptr(a), _ptr(b), _ptr(c),
                                          _stream_handle(stream, a.device)), "bn_batch_execute")
        return c

    def close(self):
        if self._h:
            _check(self._lib.bn_batch_destroy(self._h), "bn_batch_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A bn_server: continuous batching of device-resident requests."""

    def __init__(self, pool_bytes: int = 0, max_inflight: int = 0, max_batch: int = 0,
                 sequential: bool = False):
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        cfg = bn_server_config(pool_bytes, max_inflight, max_batch,
                               BN_SERVER_SEQUENTIAL if sequential else 0, 0)
        _check(lib.bn_server_create(ctypes.byref(self._h), ctypes.byref(cfg)), "bn_server_create")

    def now_us(self) -> float:
        return self._lib.bn_server_now_us(self._h)

    def submit(self, reqs: np.ndarray) -> np.ndarray:
        """Enqueue requests (REQUEST_DTYPE); returns their tickets."""
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
        tickets = np.empty(reqs.shape[0], np.uint64)
        _check(self._lib.bn_server_submit(self._h, ctypes.c_void_p(reqs.ctypes.data), reqs.shape[0],
                                          ctypes.c_void_p(tickets.ctypes.data)), "bn_server_submit")
        return tickets

    def poll(self, max_items: int = 1 << 16) -> np.ndarray:
        out = np.empty(max_items, COMPLETION_DTYPE)
        n = ctypes.c_uint32()
        _check(self._lib.bn_server_poll(self._h, ctypes.c_void_p(out.ctypes.data), max_items,
                                        ctypes.byref(n)), "bn_server_poll")
        return out[: n.value]

    def release(self, tickets) -> None:
        t = np.ascontiguousarray(tickets, dtype=np.uint64)
        _check(self._lib.bn_server_release(self._h, ctypes.c_void_p(t.ctypes.data), t.shape[0]),
               "bn_server_release")

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(self._lib.bn_server_drain(self._h, timeout_s), "bn_server_drain")

    @property
    def stats(self) -> dict:
        st = bn_server_stats()
        _check(self._lib.bn_server_get_stats(self._h, ctypes.byref(st)), "bn_server_get_stats")
        return {k: getattr(st, k) for k, _ in bn_server_stats._fields_ if k != "reserved"}

    def close(self):
        if self._h:
            _check(self._lib.bn_server_destroy(self._h), "bn_server_destroy")
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def device_to_host(ptr: int, limbs: int) -> np.ndarray:
    """Copy `limbs` u32 words at a raw device address (e.g. a completion's
    result) into a new numpy array, through the CUDA runtime the library uses."""
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("libcudart.so.13")
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _cudart.cudaMemcpy.restype = ctypes.c_int
    out = np.empty(limbs, np.uint32)
    rc = _cudart.cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr), 4 * limbs, 2)
    if rc != 0:
        raise RuntimeError(f"cudaMemcpy failed ({rc})")
    return out


_cudart = None

