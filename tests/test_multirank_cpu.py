"""The benchmark's multi-rank host logic on CPU: two gloo ranks (127.0.0.1)
run the same barrier and max-over-ranks reduction bench.py uses under
torchrun, and the whole-job value aggregates the per-rank work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    elapsed = 10.0 + 5.0 * rank                  # the slower rank decides
    m = bench.allreduce_max(elapsed, world, "cpu")
    q.put((rank, m, bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    assert [g[1] for g in got] == [15.0, 15.0]
    assert [g[2] for g in got] == [(0, 2, 0), (1, 2, 1)]


def test_weak_scaling_value():
    import bench
    # 100 multiplications per rank per step, 4 steps, slowest rank 2 ms, 8 ranks.
    assert bench.aggregate_value(100, 4, 2.0, 8) == pytest.approx(8 * 100 * 4 / 2e-3)
    assert bench.aggregate_value(100, 4, 2.0, 1) == pytest.approx(100 * 4 / 2e-3)
