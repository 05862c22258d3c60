"""Parity of bn_mul_quad (Section 3) with the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 2), (2, 1), (3, 3), (4, 4), (5, 7), (8, 8), (17, 15), (31, 32), (32, 32),
          (33, 33), (64, 64), (65, 63), (100, 3), (3, 100), (128, 128), (129, 130), (256, 256),
          (500, 20), (20, 500), (777, 1000), (1024, 1024), (2048, 2048), (4096, 4096),
          (4095, 4097), (8192, 32), (8192, 8192)]


@pytest.mark.parametrize("na,nb", SHAPES)
def test_quad_matches_oracle(na, nb):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 41 if max(na, nb) <= 2048 else 9
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(6, na * 7 + nb))
    got = to_host(bn.bn_mul_quad(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.mul(a, b), f"quad {na}x{nb}")


@pytest.mark.parametrize("q", [4, 8])
@pytest.mark.parametrize("na,nb", [(32, 32), (96, 40), (512, 512), (1000, 1000)])
def test_quad_window_sizes(q, na, nb):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(23, na, nb, seed=workloads.seed_for(6, 5000 + na + q))
    with bn.Plan(bn.BN_OP_MUL_QUAD, na, nb, 23, limbs_per_thread=q) as plan:
        got = to_host(plan.execute(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.mul(a, b), f"quad q={q} {na}x{nb}")


def test_quad_tiny_workload():
    """4096 pairs of 4096-bit integers with 5% edge cases -> 256-limb products."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.tiny_workload()
    got = to_host(bn.bn_mul_quad(to_dev(a), to_dev(b)))
    assert got.shape == (4096, 256)
    assert_limbs_equal(got, oracle.mul(a, b), "quad tiny")


def test_quad_closed_forms():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    for n in [1, 7, 32, 1000, 8192]:
        ones = np.full((2, n), 0xFFFFFFFF, np.uint32)
        got = to_host(bn.bn_mul_quad(to_dev(ones), to_dev(ones)))
        want = np.zeros((2, 2 * n), np.uint32)
        want[:, 0] = 1
        want[:, n] = 0xFFFFFFFE
        want[:, n + 1:] = 0xFFFFFFFF
        assert_limbs_equal(got, want, f"(2^N-1)^2 n={n}")


@pytest.mark.parametrize("n", [33, 4096])
def test_quad_unaligned_rows(n):
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(12, n, seed=workloads.seed_for(6, 900 + n))
    ta = torch.empty(12 * n + 1, dtype=torch.int32, device="cuda")[1:].view(12, n)
    ta.copy_(to_dev(a))
    out = torch.empty(12 * 2 * n + 1, dtype=torch.int32, device="cuda")[1:].view(12, 2 * n)
    got = to_host(bn.bn_mul_quad(ta, to_dev(b), out=out))
    assert_limbs_equal(got, oracle.mul(a, b), "quad unaligned")


@pytest.mark.parametrize("point", workloads.sweep_points(), ids=lambda p: f"{p.bits}b")
def test_quad_full_size_sampled(point):
    """Full size-sweep batches (64 MiB per side) in the benchmark's launch
    configuration; sampled rows against the oracle."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(point.batch, point.limbs, seed=point.seed, edges=True)
    got = to_host(bn.bn_mul_quad(to_dev(a), to_dev(b)))
    k = 24 if point.limbs <= 1024 else 6
    rows = np.random.default_rng(point.seed).choice(point.batch, k, replace=False)
    rows = np.union1d(rows, [19, 39, point.batch - 1])
    assert_limbs_equal(got[rows], oracle.mul(a[rows], b[rows]), f"quad {point.bits} sampled")


LANE_SHAPES = [(1, 1), (1, 2), (3, 3), (4, 4), (5, 7), (8, 8), (9, 9), (17, 15), (31, 32), (32, 32),
               (33, 33), (24, 40), (64, 64), (65, 63), (100, 3), (3, 100), (64, 1), (128, 128), (127, 1)]


@pytest.mark.parametrize("batch", [1, 37, 5000])
@pytest.mark.parametrize("na,nb", LANE_SHAPES)
def test_quad_lane_form(na, nb, batch):
    """One product per thread (variant 3): every size it holds, batches that
    fill one lane, part of a warp, and many warps with a ragged last one."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(6, 7000 + 3 * na + nb + batch))
    a[0] = 0xFFFFFFFF
    b[0] = 0xFFFFFFFF
    with bn.Plan(bn.BN_OP_MUL_QUAD, na, nb, batch, variant=3) as plan:
        got = to_host(plan.execute(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.mul(a, b), f"quad lane {na}x{nb} batch {batch}")


@pytest.mark.parametrize("na,nb", [(32, 32), (12, 20), (33, 7)])
def test_quad_lane_form_unaligned_rows(na, nb):
    """Operand and result rows off the 16-byte boundary take the word-wise staging and stores."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 70
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(6, 7500 + na + nb))
    ta = torch.empty(batch * na + 1, dtype=torch.int32, device="cuda")[1:].view(batch, na)
    ta.copy_(to_dev(a))
    out = torch.empty(batch * (na + nb) + 1, dtype=torch.int32, device="cuda")[1:].view(batch, na + nb)
    with bn.Plan(bn.BN_OP_MUL_QUAD, na, nb, batch, variant=3) as plan:
        got = to_host(plan.execute(ta, to_dev(b), out=out))
    assert_limbs_equal(got, oracle.mul(a, b), f"quad lane unaligned {na}x{nb}")


def test_quad_lane_form_limits():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    with pytest.raises(bn.BnError):
        bn.Plan(bn.BN_OP_MUL_QUAD, 129, 8, 4, variant=3)
    with pytest.raises(bn.BnError):
        bn.Plan(bn.BN_OP_MUL_QUAD, 32, 32, 4, variant=3, limbs_per_thread=4)
