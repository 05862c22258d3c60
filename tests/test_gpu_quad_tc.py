"""Parity of bn_mul_quad_tc (Section 3's column sums computed on bytes as an
exact fp16 contraction on the tensor cores) with the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

# 32 limbs = one 128-byte block; 8192 limbs of output = one tile of 256 blocks.
# Outputs wider than one tile use the circular D (the longer operand's blocks
# as D's columns): (4097, 4097) onwards, incl. lengths that are not a multiple
# of 16 blocks (4500: 141 blocks, 6000: 188, 8000: 250) and a one-block operand.
SHAPES = [(1, 1), (1, 2), (2, 1), (3, 5), (31, 33), (32, 32), (33, 31), (64, 64), (100, 3),
          (3, 100), (128, 128), (129, 130), (500, 20), (777, 1000), (1024, 1024), (2047, 2049),
          (2048, 2048), (4096, 4096), (4097, 4000), (5000, 3001), (8192, 8192), (8192, 1),
          (1, 8192), (8192, 100), (100, 8192), (4097, 4097), (4500, 4500), (6000, 5000),
          (8000, 300), (8191, 8191), (8192, 4097), (7777, 8000), (8192, 32), (8192, 33),
          # up to 64 blocks: the Toeplitz-rows form, one chunk (<= 32 blocks) or two (64 blocks)
          (2048, 1), (1, 2048), (1500, 1500), (1025, 1023), (1000, 2048), (2048, 2047), (2000, 64)]


def _tc(a, b):
    import paper_2405_14642_gb300 as bn
    got = to_host(bn.bn_mul_quad_tc(to_dev(a), to_dev(b)))
    bn.bn_tc_check()
    return got


@pytest.mark.parametrize("na,nb", SHAPES)
def test_quad_tc_matches_oracle(na, nb):
    torch_cuda()
    batch = 37 if max(na, nb) <= 2048 else 7
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(9, na * 7 + nb))
    assert_limbs_equal(_tc(a, b), oracle.mul(a, b), f"quad_tc {na}x{nb}")


def test_quad_tc_closed_forms():
    """(2^N - 1)^2: every byte 255, so every MMA sum is at its maximum
    128 * 255^2 < 2^23 and the column sums and carries are the largest."""
    torch_cuda()
    for n in [1, 7, 32, 33, 1000, 4096, 8192]:
        ones = np.full((2, n), 0xFFFFFFFF, np.uint32)
        want = np.zeros((2, 2 * n), np.uint32)
        want[:, 0] = 1
        want[:, n] = 0xFFFFFFFE
        want[:, n + 1:] = 0xFFFFFFFF
        assert_limbs_equal(_tc(ones, ones), want, f"(2^N-1)^2 n={n}")


def test_quad_tc_edges_and_many_ctas():
    """More pairs than CTAs (each CTA loops over instances, reusing its tensor
    memory and mbarriers), with the 5% edge cases, through a plan."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(700, 300, 260, seed=workloads.seed_for(9, 77), edges=True)
    with bn.Plan(bn.BN_OP_MUL_QUAD_TC, 300, 260, 700) as plan:
        assert plan.op == bn.BN_OP_MUL_QUAD_TC
        assert plan.scratch_bytes > 0
        got = to_host(plan.execute(to_dev(a), to_dev(b)))
    bn.bn_tc_check()
    assert_limbs_equal(got, oracle.mul(a, b), "quad_tc plan 700 x 300x260")


def test_quad_tc_equals_integer_schoolbook():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    for na, nb in [(4096, 4096), (3000, 1234)]:
        a, b = workloads.pair_batch(300, na, nb, seed=workloads.seed_for(9, na + nb))
        da, db = to_dev(a), to_dev(b)
        assert_limbs_equal(_tc(a, b), to_host(bn.bn_mul_quad(da, db)), f"tc vs quad {na}x{nb}")


@pytest.mark.parametrize("bits", [16384, 65536, 262144])
def test_quad_tc_full_size_sampled(bits):
    """A size-sweep batch (64 MiB per side), launched as the benchmark launches
    it, checked against the oracle on sampled rows."""
    torch_cuda()
    p = [q for q in workloads.sweep_points() if q.bits == bits][0]
    a, b = workloads.pair_batch(p.batch, p.limbs, seed=p.seed, edges=True)
    got = _tc(a, b)
    rows = np.union1d(np.random.default_rng(bits).choice(p.batch, 5, replace=False), [19, 39])
    assert_limbs_equal(got[rows], oracle.mul(a[rows], b[rows]), f"quad_tc {bits} sampled")


def test_quad_tc_errors():
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    big = torch.zeros((1, 8193), dtype=torch.int32, device="cuda")
    one = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(bn.BnError):
        bn.bn_mul_quad_tc(big, one)
    with pytest.raises(bn.BnError):
        bn.Plan(bn.BN_OP_MUL_QUAD_TC, 64, 64, 4, limbs_per_thread=4)
    x = torch.zeros((2, 16), dtype=torch.int32, device="cuda")
    out = torch.zeros((2, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(bn.BnError):
        bn.bn_mul_quad_tc(out.view(-1)[:32].view(2, 16), x, out=out)  # result overlaps an operand
    empty = torch.zeros((0, 16), dtype=torch.int32, device="cuda")
    assert bn.bn_mul_quad_tc(empty, empty).shape == (0, 32)
    bn.bn_tc_check()


def test_tc_bounded_wait_gives_up():
    """A wait with no arrival coming gives up after its limit, a second waiter
    watching the abort flag gives up with it, and the device flag reports it."""
    import time
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    t0 = time.perf_counter()
    status = bn.bn_tc_wait_selftest(20000)  # 20 ms
    elapsed = time.perf_counter() - t0
    assert status == bn.BN_ETIMEOUT
    assert elapsed < 5.0  # not the second waiter's own 10 s limit
    bn.bn_tc_check()      # the self-test leaves the flag clear


def test_mma_probe_runs_and_checks_arguments():
    """The tensor-core chain probe (bn_probe.h) completes within its bounded
    wait and refuses shapes that do not fit tensor memory or the MMA."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n, chains, chain_len in [(32, 8, 8), (64, 4, 1000), (256, 2, 3), (16, 1, 1)]:
        bn.bn_probe_mma_throughput(n, chains, chain_len, 300, 4, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for bad in [(64, 16, 8), (24, 1, 8), (272, 1, 8), (32, 0, 8), (32, 1, 0)]:
        with pytest.raises(bn.BnError):
            bn.bn_probe_mma_throughput(*bad, 10, 1, status)


@pytest.mark.parametrize("batch", [1, 2, 151, 152, 153, 305])
@pytest.mark.parametrize("na,nb", [(1024, 1024), (2048, 1500), (500, 20), (4096, 4000)])
def test_quad_tc_batch_around_the_grid(batch, na, nb):
    """Batches of one pair, around one pair per SM (152) and past two, at
    32- and 64-column slots of the Toeplitz-window kernel (each CTA fetches its
    next pair's rows ahead, so the last pair of a CTA, a CTA without a second
    pair and a grid smaller than the SM count all occur) and at 128K bits."""
    torch_cuda()
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(9, 9000 + batch * 5 + na), edges=True)
    assert_limbs_equal(_tc(a, b), oracle.mul(a, b), f"quad_tc batch {batch} {na}x{nb}")
