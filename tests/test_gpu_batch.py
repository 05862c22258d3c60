"""Mixed-size batches (bn_batch_*): every item of a batch equals the oracle,
bit for bit, in the graph form, the plain per-item form, the padded
per-class plain form and after autotuning."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu


def check_items(items, a, b, c, sample=None):
    idx = range(items.shape[0]) if sample is None else sample
    for i in idx:
        it = items[i]
        na, nb = int(it["na"]), int(it["nb"])
        ra = a[int(it["a_offset"]):int(it["a_offset"]) + na][None]
        rb = b[int(it["b_offset"]):int(it["b_offset"]) + nb][None]
        if int(it["op"]) == 0:
            want = oracle.add(ra, rb, threads=1)[0]
        else:
            want = oracle.mul(ra, rb, threads=1)[0]
        got = c[int(it["c_offset"]):int(it["c_offset"]) + want.size]
        assert_limbs_equal(got[None], want[None], f"item {i} op {int(it['op'])} {na}x{nb}")


def run(items, a, b, c_limbs, flags=0):
    import torch
    import paper_2405_14642_gb300 as bn
    ta, tb = to_dev(a), to_dev(b)
    tc = torch.full((c_limbs,), -1, dtype=torch.int32, device="cuda")
    with bn.Batch(items, flags) as batch:
        batch.execute(ta, tb, tc)
        info = batch.info
    return to_host(tc), info


@pytest.mark.parametrize("flags", [0, 2, 4, 1], ids=["graph", "plain", "plain_classes", "autotune"])
def test_mixed_small_sizes_all_items(flags):
    torch_cuda()
    items, a, b, c_limbs = workloads.mixed_workload(700, seed=workloads.seed_for(3, 1), lo=1, hi=700)
    c, info = run(items, a, b, c_limbs, flags)
    assert (info["items_add"] + info["items_quad"] + info["items_ntt64"] + info["items_crt"]
            + info["items_ntt3"]) == 700
    check_items(items, a, b, c)


@pytest.mark.parametrize("flags", [0, 4], ids=["graph", "plain_classes"])
@pytest.mark.parametrize("op", [1, 2, 3], ids=["quad", "ntt64", "crt"])
def test_forced_kinds(op, flags):
    torch_cuda()
    items, a, b, c_limbs = workloads.mixed_workload(150, seed=workloads.seed_for(3, 10 + op), lo=3,
                                                    hi=3000, mul_frac=1.0, mul_op=op)
    c, info = run(items, a, b, c_limbs, flags)
    key = {1: "items_quad", 2: "items_ntt64", 3: "items_crt"}[op]
    assert info[key] == 150
    check_items(items, a, b, c)


def test_full_range_sampled_and_plain_equals_graph():
    """Sizes log-uniform over 32..8192 limbs (the paper's whole range): the
    graph, the plain per-item form and the padded per-class form give
    identical results; sampled items and every 20th (edge-case) item against
    the oracle."""
    torch_cuda()
    items, a, b, c_limbs = workloads.mixed_workload(1500, seed=workloads.seed_for(3, 2))
    c_graph, info = run(items, a, b, c_limbs)
    c_plain, info_p = run(items, a, b, c_limbs, flags=2)
    c_cls, info_c = run(items, a, b, c_limbs, flags=4)
    assert np.array_equal(c_graph, c_plain)
    assert np.array_equal(c_graph, c_cls)
    assert info["launches"] == info["classes"] and info_p["launches"] == 1500
    assert info_c["launches"] == 3 * info_c["classes"]
    rng = np.random.default_rng(5)
    sample = np.union1d(rng.choice(1500, 60, replace=False), np.arange(19, 1500, 20)[:40])
    check_items(items, a, b, c_graph, sample)


@pytest.mark.parametrize("flags", [0, 2, 4, 1], ids=["graph", "plain", "plain_classes", "autotune"])
def test_auto_large_products_take_three_primes(flags):
    """Products of 1024..8192 limbs: the cost model sends them to the
    three-prime transform (the fastest form there), with exact results."""
    torch_cuda()
    items, a, b, c_limbs = workloads.mixed_workload(120, seed=workloads.seed_for(3, 30), lo=1024,
                                                    hi=8192, mul_frac=1.0)
    c, info = run(items, a, b, c_limbs, flags)
    assert info["items_ntt3"] > 60, info
    assert info["items_ntt3"] + info["items_quad"] + info["items_ntt64"] + info["items_crt"] == 120
    check_items(items, a, b, c)


def test_rebinding_buffers():
    """One batch, two executions on different flat arrays."""
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    items, a, b, c_limbs = workloads.mixed_workload(200, seed=workloads.seed_for(3, 3), lo=2, hi=400)
    _, a2, b2, _ = workloads.mixed_workload(200, seed=workloads.seed_for(3, 3), lo=2, hi=400,
                                            edges=False)
    a2 = a2[::-1].copy()
    with bn.Batch(items) as batch:
        for aa, bb in ((a, b), (a2, b2)):
            tc = torch.zeros(c_limbs, dtype=torch.int32, device="cuda")
            batch.execute(to_dev(aa), to_dev(bb), tc)
            check_items(items, aa, bb, to_host(tc))


def test_batch_rejects_bad_items():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    items = np.zeros(2, bn.BATCH_ITEM_DTYPE)
    items["na"] = [4, 0]
    items["nb"] = [4, 4]
    with pytest.raises(bn.BnError) as e:
        bn.Batch(items)
    assert e.value.status == 1
    items["na"] = [4, bn.BN_MUL_MAX_LIMBS + 1]
    items["op"] = 4
    with pytest.raises(bn.BnError) as e:
        bn.Batch(items)
    assert e.value.status == 4
    empty = np.zeros(0, bn.BATCH_ITEM_DTYPE)
    with bn.Batch(empty) as batch:
        assert batch.info["classes"] == 0
    with bn.Batch(empty, bn.BN_BATCH_PLAIN_CLASSES) as batch:
        assert batch.info["launches"] == 0
    items["na"] = [4, 4]
    with pytest.raises(bn.BnError) as e:
        bn.Batch(items, bn.BN_BATCH_PLAIN | bn.BN_BATCH_PLAIN_CLASSES)
    assert e.value.status == 1
