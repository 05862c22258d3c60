"""The debug build (compiled with BN_DEBUG): on small shapes of every product
form (integer and tensor-core schoolbook, one- and two-prime transforms
unsplit and split over a two-CTA cluster, three primes), called through the
C ABI of the debug library, the checks for words or carries beyond na + nb
(Section 3.2, Fig. 5) and for shared-memory indices out of range must leave
the error word at zero, and every product must equal the oracle's."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import _build, workloads

pytestmark = pytest.mark.gpu

SHAPES = {
    "bn_mul_quad": [(1, 1, 5), (7, 3, 9), (33, 17, 20), (128, 128, 41), (513, 257, 6), (1000, 999, 4),
                    (32, 32, 4864), (64, 9, 5000), (13, 6, 4900)],             # the last three: one per thread
    "bn_mul_quad_tc": [(1, 1, 5), (100, 37, 7), (1024, 1024, 3), (1500, 700, 3), (2048, 2048, 3), (4224, 100, 2)],
    "bn_mul_ntt3": [(5, 3, 9), (512, 512, 6), (8192, 8192, 2)],
    "ntt64": [(3, 2, 9), (500, 600, 7), (3000, 2500, 3), (8192, 8192, 2)],      # unsplit, S = 2, S = 4
    "crt": [(3, 2, 9), (1024, 1024, 5), (8192, 5000, 2), (8192, 8192, 2)],      # unsplit, S = 2
}


@pytest.fixture(scope="module")
def dbg():
    torch_cuda()
    lib = ctypes.CDLL(str(_build.build(debug=True)))
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    for name in ("bn_mul_quad", "bn_mul_quad_tc", "bn_mul_ntt3"):
        getattr(lib, name).argtypes = [vp, vp, vp, u32, u32, u64, vp]
    lib.bn_mul_ntt.argtypes = [vp, vp, vp, u32, u32, u64, ctypes.c_int, vp]
    lib.bn_debug_word.restype = ctypes.c_uint32
    assert lib.bn_debug_build() == 1
    assert lib.bn_debug_word() == 0
    return lib


def run(lib, form, a, b):
    import torch
    ta, tb = to_dev(a), to_dev(b)
    batch, na, nb = a.shape[0], a.shape[1], b.shape[1]
    tc = torch.full((batch, na + nb), -1, dtype=torch.int32, device="cuda")
    ptrs = (ctypes.c_void_p(ta.data_ptr()), ctypes.c_void_p(tb.data_ptr()), ctypes.c_void_p(tc.data_ptr()))
    if form in ("ntt64", "crt"):
        st = lib.bn_mul_ntt(*ptrs, na, nb, batch, int(form == "crt"), None)
    else:
        st = getattr(lib, form)(*ptrs, na, nb, batch, None)
    assert st == 0, (form, st)
    torch.cuda.synchronize()
    return to_host(tc)


@pytest.mark.parametrize("form", sorted(SHAPES))
def test_debug_checks_stay_clear(dbg, form):
    for na, nb, batch in SHAPES[form]:
        a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(11, na + 3 * nb))
        a[0] = 0xFFFFFFFF          # all-ones operands: the largest products and longest carries
        b[0] = 0xFFFFFFFF
        got = run(dbg, form, a, b)
        word = dbg.bn_debug_word()
        assert word == 0, f"{form} {na}x{nb}: debug bits {word:#x}"
        assert_limbs_equal(got, oracle.mul(a, b), f"{form} {na}x{nb} (debug build)")


def test_regular_build_reports_no_checks():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    lib = bn.load()
    lib.bn_debug_word.restype = ctypes.c_uint32
    assert lib.bn_debug_build() == 0 and lib.bn_debug_word() == 0
