"""Parity of bn_mul_ntt3 (Section 4's transform product over three 32-bit
primes with 32-bit digits and Garner recombination) with the CPU oracle, bit
for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (8, 8), (31, 33), (32, 32), (100, 3), (3, 100),
          (128, 128), (129, 130), (500, 20), (777, 1000), (1024, 1024), (2048, 2048),
          (2049, 2047), (4096, 4096), (4097, 4000), (8192, 8192), (8192, 1), (1, 8192)]


@pytest.mark.parametrize("na,nb", SHAPES)
def test_ntt3_matches_oracle(na, nb):
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 37 if max(na, nb) <= 2048 else 7
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(8, na * 7 + nb))
    got = to_host(bn.bn_mul_ntt3(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.mul(a, b), f"ntt3 {na}x{nb}")


def test_ntt3_closed_forms():
    """(2^N - 1)^2: every coefficient at its maximum, the longest carry chains."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    for n in [1, 7, 32, 1000, 4096, 8192]:
        ones = np.full((2, n), 0xFFFFFFFF, np.uint32)
        got = to_host(bn.bn_mul_ntt3(to_dev(ones), to_dev(ones)))
        want = np.zeros((2, 2 * n), np.uint32)
        want[:, 0] = 1
        want[:, n] = 0xFFFFFFFE
        want[:, n + 1:] = 0xFFFFFFFF
        assert_limbs_equal(got, want, f"(2^N-1)^2 n={n}")


def test_ntt3_many_ctas_and_plan():
    """More pairs than resident CTAs (the persistent grid loops), through a plan,
    with the 5% edge cases; also the plan's transform length and scratch."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(1500, 256, 256, seed=workloads.seed_for(8, 99))
    with bn.Plan(bn.BN_OP_MUL_NTT3, 256, 256, 1500) as plan:
        assert plan.transform_length == 512
        assert plan.scratch_bytes > 0
        got = to_host(plan.execute(to_dev(a), to_dev(b)))
    assert_limbs_equal(got, oracle.mul(a, b), "ntt3 plan 1500 x 256")


def test_ntt3_full_size_sampled():
    """The 256K-bit sweep batch (2048 pairs, 64 MiB per side), as the benchmark
    launches it, checked on sampled rows."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    p = [q for q in workloads.sweep_points() if q.bits == 262144][0]
    a, b = workloads.pair_batch(p.batch, p.limbs, seed=p.seed, edges=False)
    got = to_host(bn.bn_mul_ntt3(to_dev(a), to_dev(b)))
    rows = np.random.default_rng(5).choice(p.batch, 6, replace=False)
    assert_limbs_equal(got[rows], oracle.mul(a[rows], b[rows]), "ntt3 256K sampled")


def test_ntt3_equals_other_transforms():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(19, 700, 333, seed=workloads.seed_for(8, 123))
    da, db = to_dev(a), to_dev(b)
    got = to_host(bn.bn_mul_ntt3(da, db))
    assert_limbs_equal(got, to_host(bn.bn_mul_ntt(da, db, crt=True)), "ntt3 vs crt")
    assert_limbs_equal(got, to_host(bn.bn_mul_quad(da, db)), "ntt3 vs quad")


def test_ntt3_rejects_batch_items_and_oversize():
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    with pytest.raises(bn.BnError):
        bn.Plan(bn.BN_OP_MUL_NTT3, 8193, 8, 1)
    items = np.zeros(1, bn.BATCH_ITEM_DTYPE)
    items["op"], items["na"], items["nb"] = bn.BN_OP_MUL_NTT3, 4, 4
    with pytest.raises(bn.BnError):
        bn.Batch(items)
    x = torch.zeros((2, 4), dtype=torch.int32, device="cuda")
    empty = torch.zeros((0, 4), dtype=torch.int32, device="cuda")
    assert bn.bn_mul_ntt3(empty, empty).shape == (0, 8)
    assert to_host(bn.bn_mul_ntt3(x, x)).sum() == 0


def test_host_async_plans_on_streams():
    """bn_plan_execute_host_async: three plans of different ops on three
    streams with pinned host buffers, enqueued back to back, each result equal
    to the oracle once the streams are synchronised."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    cases = [(bn.BN_OP_MUL_NTT3, 600, 500), (bn.BN_OP_MUL_QUAD, 300, 77), (bn.BN_OP_ADD, 1000, 999)]
    streams = [torch.cuda.Stream() for _ in cases]
    runs = []
    for k, (op, na, nb) in enumerate(cases):
        a, b = workloads.pair_batch(33, na, nb, seed=workloads.seed_for(8, 500 + k))
        plan = bn.Plan(op, na, nb, 33)
        pa = torch.from_numpy(a.view(np.int32)).pin_memory()
        pb = torch.from_numpy(b.view(np.int32)).pin_memory()
        pc = torch.empty((33, plan.out_limbs), dtype=torch.int32).pin_memory()
        runs.append((op, a, b, plan, pa, pb, pc))
    for rep in range(2):
        for (op, a, b, plan, pa, pb, pc), st in zip(runs, streams):
            pc.fill_(-1)
            plan.execute_host_async(pa, pb, pc, stream=st)
        torch.cuda.synchronize()
        for op, a, b, plan, pa, pb, pc in runs:
            want = oracle.add(a, b) if op == bn.BN_OP_ADD else oracle.mul(a, b)
            assert_limbs_equal(pc.numpy().view(np.uint32), want, f"async op {op} rep {rep}")
    for run in runs:
        run[3].close()
    with bn.Plan(bn.BN_OP_ADD, 4, 4, 2) as plan:
        with pytest.raises(TypeError):
            plan.execute_host_async(np.zeros((2, 4), np.uint32), np.zeros((2, 4), np.uint32),
                                    np.zeros((2, 5), np.uint32))


@pytest.mark.parametrize("na,nb,kind", [(64, 64, "quad"), (256, 200, "quad"), (8192, 1, "quad"),
                                        (1024, 1024, "ntt3"), (4096, 3000, "ntt3"), (8192, 8192, "ntt3")])
def test_auto_plans_and_bn_mul(na, nb, kind):
    """BN_OP_MUL_AUTO plans resolve to the cost model's product (schoolbook for
    small operands, three primes from 8K bits) and bn_mul equals the oracle."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    batch = 9 if max(na, nb) > 2048 else 31
    a, b = workloads.pair_batch(batch, na, nb, seed=workloads.seed_for(8, 700 + na + nb))
    with bn.Plan(bn.BN_OP_MUL_AUTO, na, nb, batch) as plan:
        want_op = bn.BN_OP_MUL_QUAD if kind == "quad" else bn.BN_OP_MUL_NTT3
        assert plan.op == want_op and plan.out_limbs == na + nb
        got_plan = to_host(plan.execute(to_dev(a), to_dev(b)))
    got = to_host(bn.bn_mul(to_dev(a), to_dev(b)))
    want = oracle.mul(a, b)
    assert_limbs_equal(got, want, f"bn_mul {na}x{nb}")
    assert_limbs_equal(got_plan, want, f"auto plan {na}x{nb}")
