"""Serving loop (bn_server_*): requests submitted while others are on the GPU
are batched continuously; every result equals the same request computed alone
(and the oracle), bit for bit."""
import time

import numpy as np
import pytest

import oracle
from gpu_util import to_dev, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu


def make_requests(bn, count, seed, lo=1, hi=1500, mul_frac=0.85):
    items, a, b, _ = workloads.mixed_workload(count, seed=seed, lo=lo, hi=hi, mul_frac=mul_frac)
    ta, tb = to_dev(a), to_dev(b)
    reqs = np.zeros(count, bn.REQUEST_DTYPE)
    reqs["op"] = items["op"]
    reqs["na"] = items["na"]
    reqs["nb"] = items["nb"]
    reqs["a"] = ta.data_ptr() + 4 * items["a_offset"].astype(np.uint64)
    reqs["b"] = tb.data_ptr() + 4 * items["b_offset"].astype(np.uint64)
    reqs["arrival_us"] = -1.0
    return reqs, items, a, b, (ta, tb)


def expected(items, a, b, i):
    it = items[i]
    ra = a[int(it["a_offset"]):int(it["a_offset"]) + int(it["na"])][None]
    rb = b[int(it["b_offset"]):int(it["b_offset"]) + int(it["nb"])][None]
    return (oracle.add if int(it["op"]) == 0 else oracle.mul)(ra, rb, threads=1)[0]


def run_server(bn, reqs, chunks=8, gap_s=0.002, release=True, **cfg):
    results = {}
    with bn.Server(**cfg) as srv:
        tickets = []
        for part in np.array_split(np.arange(reqs.shape[0]), chunks):
            tickets.extend(srv.submit(reqs[part]).tolist())
            time.sleep(gap_s)                        # later requests arrive while earlier run
            for comp in srv.poll():
                results[int(comp["ticket"])] = bn.device_to_host(int(comp["c"]), int(comp["limbs"]))
                if release:
                    srv.release([comp["ticket"]])
        deadline = time.time() + 60
        while len(results) < len(tickets) and time.time() < deadline:
            for comp in srv.poll():
                results[int(comp["ticket"])] = bn.device_to_host(int(comp["c"]), int(comp["limbs"]))
                if release:
                    srv.release([comp["ticket"]])
            time.sleep(0.001)
        stats = srv.stats
    return [results.get(t) for t in tickets], stats


def test_mixed_results_equal_alone_and_oracle():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    reqs, items, a, b, keep = make_requests(bn, 900, workloads.seed_for(4, 1))
    got, stats = run_server(bn, reqs, max_inflight=3, max_batch=128)
    assert stats["completed"] == 900 and stats["batches"] > 1
    alone, _ = run_server(bn, reqs, chunks=1, sequential=True)
    for i in range(900):
        assert got[i] is not None
        assert np.array_equal(got[i], alone[i]), f"request {i}: mix != alone"
        assert np.array_equal(got[i], expected(items, a, b, i)), f"request {i}: != oracle"


def test_admission_by_pool_budget():
    """A pool far smaller than the total of the results: requests wait for
    released results and still all complete correctly."""
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    reqs, items, a, b, keep = make_requests(bn, 300, workloads.seed_for(4, 2), lo=64, hi=2000)
    total = int(((reqs["na"] + reqs["nb"]) * 4).sum())
    got, stats = run_server(bn, reqs, chunks=3, pool_bytes=64 << 10, max_inflight=2, max_batch=64)
    assert total > 10 * (64 << 10) and stats["pool_high_water"] <= 64 << 10
    for i in range(0, 300, 7):
        assert np.array_equal(got[i], expected(items, a, b, i))


def test_drain_times_out_when_results_are_never_released():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    reqs, *_ , keep = make_requests(bn, 40, workloads.seed_for(4, 3), lo=256, hi=512, mul_frac=1.0)
    with bn.Server(pool_bytes=16 << 10, max_inflight=1, max_batch=4) as srv:
        srv.submit(reqs)
        with pytest.raises(bn.BnError) as e:
            srv.drain(timeout_s=0.5)
        assert e.value.status == 5                    # BN_ETIMEOUT
        done = srv.poll()
        assert 0 < len(done) < 40


def test_bad_requests_are_rejected():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    reqs, *_ , keep = make_requests(bn, 4, workloads.seed_for(4, 4), lo=4, hi=8)
    bad = reqs.copy()
    bad["na"][1] = 0
    with bn.Server(pool_bytes=1 << 20) as srv:
        with pytest.raises(bn.BnError) as e:
            srv.submit(bad)
        assert e.value.status == 1 and srv.stats["submitted"] == 0
        bad = reqs.copy()
        bad["a"][2] += 2                              # unaligned operand
        with pytest.raises(bn.BnError):
            srv.submit(bad)
    with pytest.raises(bn.BnError) as e:
        bn.Server(pool_bytes=(8 << 30) + 1)
    assert e.value.status == 4
