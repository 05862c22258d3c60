"""Host-side accounting of bench.py (no GPU): the workload, transform lengths,
algorithmic bytes and word products per launch."""
import bench
from paper_2405_14642_gb300 import workloads


def test_sweep_workload_shape():
    pts = workloads.sweep_points()
    assert [p.bits for p in pts] == [1 << e for e in range(10, 19)]
    for p in pts:
        assert p.limbs * 32 == p.bits
        assert p.batch * p.limbs * 4 == 64 << 20     # 64 MiB of limbs per side
    assert pts[0].batch == 524288 and pts[-1].batch == 2048


def test_transform_lengths_and_counts():
    n64, ncrt, mm64, mmcrt = bench.ntt_lengths(8192)   # 256K bits
    assert (n64, ncrt) == (32768, 16384)
    assert mm64 == 3 * 16384 * 15 + 2 * 32768
    assert mmcrt == 2 * (3 * 8192 * 14 + 2 * 16384)
    assert bench.ntt_lengths(512)[:2] == (2048, 1024)  # 16K bits


def test_ops_and_algorithmic_work():
    ops = bench.build_ops()
    labels = [o.label for o in ops]
    assert len(ops) == 9 * 2 + 5 * 3
    assert labels[:2] == ["add@1K", "quad@1K"] and labels[-2:] == ["crt@256K", "ntt3@256K"]
    add = next(o for o in ops if o.label == "add@256K")
    assert add.bytes == 4 * (3 * 8192 + 1) * 2048 and add.mults == 0
    # the schoolbook runs on the tensor cores from 16K bits up
    assert next(o for o in ops if o.label == "quad@8K").name == "quad"
    quad = next(o for o in ops if o.label == "quadtc@256K")
    assert quad.prods == 8192 * 8192 * 2048 and quad.nout == 16384
    assert [o.bits for o in ops if o.name == "quadtc"] == [1 << e for e in range(14, 19)]
    ntt = next(o for o in ops if o.label == "ntt64@256K")
    assert ntt.prods == 4 * bench.ntt_lengths(8192)[2] * 2048
    # three primes of 32 bits at N = 16384: 3 * (3 * 8192 * 14 + 2 * 16384) word products
    ntt3 = next(o for o in ops if o.label == "ntt3@256K")
    assert ntt3.prods == 3 * (3 * 8192 * 14 + 2 * 16384) * 2048 and ntt3.nout == 16384
    cfg = bench.workload_config(ops, 1)
    assert cfg["sizes_bits"][-1] == 262144 and cfg["batch_per_size"]["1024"] == 524288
