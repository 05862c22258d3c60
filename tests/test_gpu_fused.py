"""Parity of the same-length product and the fused programs of Section 6
(bn_mul_low, bn_poly, bn_add6) with the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import programs
from gpu_util import assert_limbs_equal, to_dev, to_host, torch_cuda
from paper_2405_14642_gb300 import workloads

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 4, 7, 8, 15, 16, 17, 31, 32, 33, 63, 64, 100, 128, 255, 256, 513, 1000,
         1024, 2047, 2048, 2049, 4096, 4100, 8191, 8192]
OPS = ["mul_low", "poly", "add6"]


def _batch(n):
    return 37 if n <= 1024 else (11 if n <= 4100 else 5)


def _run(name, a, b, **kw):
    import paper_2405_14642_gb300 as bn
    return to_host(getattr(bn, "bn_" + name)(a, b, **kw))


@pytest.mark.parametrize("name", OPS)
@pytest.mark.parametrize("n", SIZES)
def test_fused_matches_oracle(name, n):
    torch_cuda()
    a, b = workloads.pair_batch(_batch(n), n, seed=workloads.seed_for(7, n))
    got = _run(name, to_dev(a), to_dev(b))
    assert_limbs_equal(got, getattr(programs, name)(a, b), f"{name} n={n}")


@pytest.mark.parametrize("name", OPS)
@pytest.mark.parametrize("n,batch", [(4, 1000), (32, 3001), (96, 517), (2000, 70)])
def test_fused_many_ctas(name, n, batch):
    """Several instances per CTA and a ragged last CTA."""
    torch_cuda()
    a, b = workloads.pair_batch(batch, n, seed=workloads.seed_for(7, 9000 + n))
    got = _run(name, to_dev(a), to_dev(b))
    assert_limbs_equal(got, getattr(programs, name)(a, b), f"{name} n={n} batch={batch}")


@pytest.mark.parametrize("name", OPS)
@pytest.mark.parametrize("n", [8, 64, 1024])
def test_fused_unaligned_rows(name, n):
    """Operands 4 bytes off a 16-byte boundary take the 32-bit load path."""
    torch = torch_cuda()
    batch = 9
    a, b = workloads.pair_batch(batch, n, seed=workloads.seed_for(7, 7000 + n))
    fa = torch.zeros(batch * n + 1, dtype=torch.int32, device="cuda")
    fa[1:] = to_dev(a).view(-1)
    da = fa[1:].view(batch, n)
    assert da.data_ptr() % 16 != 0
    got = _run(name, da, to_dev(b))
    assert_limbs_equal(got, getattr(programs, name)(a, b), f"{name} unaligned n={n}")


@pytest.mark.parametrize("name", OPS)
def test_fused_same_operand(name):
    torch_cuda()
    a, _ = workloads.pair_batch(13, 300, seed=workloads.seed_for(7, 8000))
    da = to_dev(a)
    got = _run(name, da, da)
    assert_limbs_equal(got, getattr(programs, name)(a, a), f"{name} a == b")


def test_mul_low_is_low_half_of_quad():
    torch_cuda()
    import paper_2405_14642_gb300 as bn
    a, b = workloads.pair_batch(21, 777, seed=workloads.seed_for(7, 8001))
    full = to_host(bn.bn_mul_quad(to_dev(a), to_dev(b)))
    low = _run("mul_low", to_dev(a), to_dev(b))
    assert_limbs_equal(low, full[:, :777], "low half of quad")


def test_add6_closed_form_all_ones():
    """a = b = 2^(32n) - 1: 8a + 13b = -21 mod 2^(32n)."""
    torch_cuda()
    for n in [1, 5, 4096, 8192]:
        ones = np.full((3, n), 0xFFFFFFFF, np.uint32)
        got = _run("add6", to_dev(ones), to_dev(ones))
        want = np.full((3, n), 0xFFFFFFFF, np.uint32)
        want[:, 0] = (1 << 32) - 21
        assert_limbs_equal(got, want, f"add6 all ones n={n}")


def test_fused_errors():
    torch = torch_cuda()
    import paper_2405_14642_gb300 as bn
    a = torch.zeros((2, 8193), dtype=torch.int32, device="cuda")
    for name in OPS:
        with pytest.raises(bn.BnError):
            getattr(bn, "bn_" + name)(a, a)
    x = torch.zeros((2, 16), dtype=torch.int32, device="cuda")
    for name in OPS:
        with pytest.raises(bn.BnError):
            getattr(bn, "bn_" + name)(x, x, out=x)          # result overlaps an operand
        with pytest.raises(ValueError):
            getattr(bn, "bn_" + name)(x, x[:, :8].contiguous())
        empty = torch.zeros((0, 16), dtype=torch.int32, device="cuda")
        assert getattr(bn, "bn_" + name)(empty, empty).shape == (0, 16)


@pytest.mark.parametrize("name", OPS)
@pytest.mark.parametrize("bits", [65536, 262144])
def test_fused_full_size_sampled(name, bits):
    """The size-sweep batch (64 MiB of operands per side), launched as the
    benchmark launches it, checked against the oracle on sampled rows."""
    torch_cuda()
    p = [q for q in workloads.sweep_points() if q.bits == bits][0]
    a, b = workloads.pair_batch(p.batch, p.limbs, seed=p.seed, edges=True)
    got = _run(name, to_dev(a), to_dev(b))
    rows = np.union1d(np.random.default_rng(bits).choice(p.batch, 4, replace=False), [19, 39, 59])
    assert_limbs_equal(got[rows], getattr(programs, name)(a[rows], b[rows]), f"{name} {bits} sampled")
