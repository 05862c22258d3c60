"""Parity of bn_mul_ntt (Section 4; single 64-bit prime with 16-bit digits and
two-prime CRT with 32-bit digits) with the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (8, 8), (31, 33), (32, 32), (100, 3), (3, 100),
          (128, 128), (129, 130), (500, 20), (777, 1000), (1024, 1024), (2048, 2048),
          (2049, 2047), (4096, 4096), (4097, 4000), (8192, 8192), (8192, 1), (1, 8192)]


@pytest.mark.parametrize("crt", [False, True], ids=["ntt64", "crt"])
@pytest.mark.parametrize("na,nb", SHAPES)
def test_ntt_matches_oracle(crt, na, nb):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 37 if max(na, nb) <= 2048 else 7
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(7, na * 7 + nb))
    got = to_host(bn.bn_mul_ntt(to_dev(a), to_dev(b), crt=crt))
    assert_limbs_equal(got, oracle.mul(a, b), f"{'crt' if crt else 'ntt64'} {na}x{nb}")


@pytest.mark.parametrize("crt", [False, True], ids=["ntt64", "crt"])
def test_ntt_closed_forms(crt):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    for n in [1, 7, 32, 1000, 4096, 8192]:
        ones = np.full((2, n), 0xFFFFFFFF, np.uint32)
        got = to_host(bn.bn_mul_ntt(to_dev(ones), to_dev(ones), crt=crt))
        want = np.zeros((2, 2 * n), np.uint32)
        want[:, 0] = 1
        want[:, n] = 0xFFFFFFFE
        want[:, n + 1:] = 0xFFFFFFFF
        assert_limbs_equal(got, want, f"(2^N-1)^2 n={n}")


@pytest.mark.parametrize("crt", [False, True], ids=["ntt64", "crt"])
def test_ntt_tiny_workload(crt):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.tiny_workload()
    got = to_host(bn.bn_mul_ntt(to_dev(a), to_dev(b), crt=crt))
    assert_limbs_equal(got, oracle.mul(a, b), "ntt tiny")


def test_ntt_plan_properties():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    # 16-bit digits: N = next pow2 of 2 (na + nb); 32-bit digits: of na + nb.
    # Split transforms run on CTA clusters and hold no scratch (the two-prime
    # form keeps the first prime's coefficients in global scratch only where
    # a third shared buffer would lower occupancy).
    with bn.Plan(bn.BN_OP_MUL_NTT64, 8192, 8192, 4) as p:
        assert p.transform_length == 32768 and p.scratch_bytes == 0
    with bn.Plan(bn.BN_OP_MUL_NTT64, 512, 512, 4) as p:
        assert p.transform_length == 2048 and p.scratch_bytes == 0
    with bn.Plan(bn.BN_OP_MUL_NTT_CRT, 8192, 8192, 4) as p:
        assert p.transform_length == 16384 and p.scratch_bytes == 0
    with pytest.raises(bn.BnError) as e:
        bn.Plan(bn.BN_OP_MUL_NTT64, 8193, 16, 1)
    assert e.value.status == 4


@pytest.mark.parametrize("crt", [False, True], ids=["ntt64", "crt"])
@pytest.mark.parametrize("point", [p for p in workloads.sweep_points() if p.bits in workloads.NTT_BITS],
                         ids=lambda p: f"{p.bits}b")
def test_ntt_full_size_sampled(crt, point):
    """Full NTT-sweep batches (64 MiB per side) in the benchmark's launch
    configuration; sampled rows against the oracle."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(point.batch, point.limbs, seed=point.seed, edges=True)
    got = to_host(bn.bn_mul_ntt(to_dev(a), to_dev(b), crt=crt))
    rows = np.random.default_rng(point.seed + crt).choice(point.batch, 8, replace=False)
    rows = np.union1d(rows, [19, 39, 59, 79, 99, point.batch - 1])
    assert_limbs_equal(got[rows], oracle.mul(a[rows], b[rows]), f"ntt {point.bits} sampled")


def test_large_plan_still_launches_after_small_plan():
    """The dynamic shared-memory cap is per kernel function: creating a small
    plan after a large one must not stop the large one from launching."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(3, 1024, 1024, seed=workloads.seed_for(7, 4242))
    big = bn.Plan(bn.BN_OP_MUL_NTT64, 1024, 1024, 3)
    small = bn.Plan(bn.BN_OP_MUL_NTT64, 4, 4, 3)
    small_q = bn.Plan(bn.BN_OP_MUL_QUAD, 4, 4, 3)
    try:
        assert_limbs_equal(to_host(big.execute(to_dev(a), to_dev(b))), oracle.mul(a, b), "big")
    finally:
        for p in (big, small, small_q):
            p.close()
