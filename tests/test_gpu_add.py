"""Parity of bn_add (Section 2 carry scan) with the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (2, 3), (4, 4), (5, 7), (31, 32), (32, 32), (33, 31), (100, 3), (3, 100),
          (128, 128), (129, 130), (255, 256), (256, 256), (1000, 999), (1024, 1024),
          (4096, 4096), (4100, 4092), (8192, 8192), (16383, 16384), (16384, 16384)]


@pytest.mark.parametrize("na,nb", SHAPES)
def test_add_matches_oracle(na, nb):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 45 if max(na, nb) <= 4096 else 21
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(5, na * 7 + nb))
    got = to_host(bn.bn_add(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.add(a, b), f"add {na}x{nb}")


def test_add_tiny_workload():
    """4096 pairs of 4096-bit integers with 5% carry-chain edge cases."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.tiny_workload()
    got = to_host(bn.bn_add(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.add(a, b), "add tiny")


@pytest.mark.parametrize("n", [32, 129, 4096])
def test_add_unaligned_rows(n):
    """Operands that start 4 bytes off a 16-byte boundary take the scalar path."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(40, n, seed=workloads.seed_for(5, 900 + n))
    ta = torch.empty(40 * n + 1, dtype=torch.int32, device="cuda")[1:].view(40, n)
    tb = torch.empty(40 * n + 1, dtype=torch.int32, device="cuda")[1:].view(40, n)
    ta.copy_(to_dev(a))
    tb.copy_(to_dev(b))
    assert ta.data_ptr() % 16 != 0
    assert_limbs_equal(to_host(bn.bn_add(ta, tb)), oracle.add(a, b), "add unaligned")


@pytest.mark.parametrize("n", [2048, 4096, 8192])
def test_add_streaming_rounds(n):
    """Aligned equal-length rows of 64K-256K bits take the persistent,
    double-buffered kernel: enough instances for several rounds per CTA and
    a ragged last round, 5% carry-chain edge cases, every row checked."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 3 * 152 * 3 + 17
    a, b = workloads.pair_batch(batch, n, n, seed=workloads.seed_for(12, n))
    got = to_host(bn.bn_add(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.add(a, b), f"stream {n}")


def test_add_full_carry_chains():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    for n in [1, 4, 32, 128, 512, 8192, 16384]:
        ones = np.full((3, n), 0xFFFFFFFF, np.uint32)
        one = np.zeros((3, n), np.uint32)
        one[:, 0] = 1
        one[1, 0] = 0xFFFFFFFF
        one[2, :] = 0
        got = to_host(bn.bn_add(to_dev(ones), to_dev(one)))
        assert_limbs_equal(got, oracle.add(ones, one), f"chain {n}")


@pytest.mark.parametrize("point", workloads.sweep_points(), ids=lambda p: f"{p.bits}b")
def test_add_full_size_sampled(point):
    """The size-sweep batches at full size (64 MiB per side), in the launch
    configuration the benchmark times; 64 sampled rows against the oracle."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(point.batch, point.limbs, seed=point.seed, edges=True)
    got = to_host(bn.bn_add(to_dev(a), to_dev(b)))
    rows = np.random.default_rng(point.seed).choice(point.batch, 64, replace=False)
    rows = np.union1d(rows, [0, 19, 39, point.batch - 1])
    assert_limbs_equal(got[rows], oracle.add(a[rows], b[rows]), f"add {point.bits} sampled")


def test_add_plan_and_host_path():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(50, 300, 200, seed=workloads.seed_for(5, 77))
    want = oracle.add(a, b)
    with bn.Plan(bn.BN_OP_ADD, 300, 200, 50) as plan:
        assert plan.out_limbs == 301
        assert_limbs_equal(to_host(plan.execute(to_dev(a), to_dev(b))), want, "plan")
        assert_limbs_equal(plan.execute_host(a, b), want, "plan host")
    with bn.Plan(bn.BN_OP_ADD, 300, 200, 50, limbs_per_thread=8, cta_threads=128) as plan:
        assert_limbs_equal(to_host(plan.execute(to_dev(a), to_dev(b))), want, "plan tuned")


def test_add_errors():
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    buf = torch.zeros(4 * 9, dtype=torch.int32, device="cuda")
    a = buf[:32].view(4, 8)
    with pytest.raises(bn.BnError) as e:            # result overlaps an operand
        bn.bn_add(a, a, out=buf.view(4, 9))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        bn.bn_add(a, a, out=torch.zeros((4, 8), dtype=torch.int32, device="cuda"))
    big = torch.zeros((1, bn.BN_ADD_MAX_LIMBS + 1), dtype=torch.int32, device="cuda")
    with pytest.raises(bn.BnError) as e:
        bn.bn_add(big, big)
    assert e.value.status == 4
    with pytest.raises(bn.BnError) as e:
        bn.Plan(bn.BN_OP_ADD, 0, 4, 1)
    assert e.value.status == 1
    empty = torch.zeros((0, 8), dtype=torch.int32, device="cuda")
    assert bn.bn_add(empty, empty).shape == (0, 9)
