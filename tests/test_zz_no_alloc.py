"""bn_mul_ntt_noalloc: the transform multiplication for callers that cannot
call cudaMalloc (their device memory belongs to another allocator, or they
cannot afford cudaMalloc's implicit device-wide synchronisation).  Its
scratch and tables live in fixed device arrays shared by every call.

Checked through the C ABI against the allocating entry point bn_mul_ntt and
against the CPU oracle, bit for bit (the tolerance of every parity test
here), on two calls in a row per case, so the second call runs on the arrays
the first one left behind.  A captured call replayed between eager calls of
other sizes must still read the tables of its own size.
Sizes include transforms that need scratch (two-prime CRT at every size, and
the split single-prime transform at 128K/256K bits).  The file sorts last so
a run that stops at the first failure has already run every other test; it
passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [(False, 4096, 4096, 12), (True, 8192, 8192, 9), (False, 8192, 8192, 70),
         (True, 100, 37, 33), (False, 513, 129, 40), (True, 2048, 2048, 300)]


@pytest.mark.parametrize("crt,na,nb,batch", CASES,
                         ids=[f"{'crt' if c else 'ntt64'}-{na}x{nb}-b{bt}" for c, na, nb, bt in CASES])
def test_noalloc_matches_allocating_entry_point(crt, na, nb, batch):
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    for call in range(2):
        a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(9, na + 31 * nb + call))
        ta, tb = to_dev(a), to_dev(b)
        want = to_host(bn.bn_mul_ntt(ta, tb, crt=crt))
        out = torch.full((batch, na + nb), -1, dtype=torch.int32, device="cuda")
        got = to_host(bn.bn_mul_ntt_noalloc(ta, tb, crt=crt, out=out))
        torch.cuda.synchronize()
        assert_limbs_equal(got, want, f"noalloc call {call} crt={crt} {na}x{nb}")
        assert_limbs_equal(got, oracle.mul(a, b), f"noalloc call {call} vs oracle")


def test_noalloc_captured_call_keeps_its_tables():
    """A call captured into a CUDA graph at one transform length, eager calls
    at another length before and after a replay: every result exact."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn

    def operands(n, seed):
        a, b = workloads.pair_batch(5, n, n, seed=workloads.seed_for(9, seed))
        return a, b, to_dev(a), to_dev(b)

    ax, bx, tax, tbx = operands(1024, 501)      # captured size
    ay, by, tay, tby = operands(96, 502)        # eager size (another transform length)
    bn.bn_mul_ntt_noalloc(tay, tby)             # device set-up before any capture
    torch.cuda.synchronize()
    out_g = torch.full((5, 2048), -1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        bn.bn_mul_ntt_noalloc(tax, tbx, out=out_g)
    want_x, want_y = oracle.mul(ax, bx), oracle.mul(ay, by)
    for rep in range(2):
        got_y = to_host(bn.bn_mul_ntt_noalloc(tay, tby))
        assert_limbs_equal(got_y, want_y, f"eager call before replay {rep}")
        out_g.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert_limbs_equal(to_host(out_g), want_x, f"replay {rep}")
    got_y = to_host(bn.bn_mul_ntt_noalloc(tay, tby))
    assert_limbs_equal(got_y, want_y, "eager call after the replays")


def test_noalloc_rejects_sizes_beyond_its_maximum():
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    big = torch.zeros((1, bn.BN_MUL_MAX_LIMBS + 1), dtype=torch.int32, device="cuda")
    small = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(bn.BnError) as e:
        bn.bn_mul_ntt_noalloc(big, small)
    assert e.value.status == 4 and "BN_NOALLOC_MAX_LIMBS" in str(e.value)
