"""The tensor-core schoolbook's formulation checked on the CPU: the column
sums of Section 3's product (Eq. 1) computed on bytes as blocks
D_J = W_J X^T with W_J[r][c] = b-byte (128 J + r - c), accumulated in f32 on a
bias of 2^23, are exact, their bit patterns give the integers back, and the
column sums carried into limbs give the product (compared with Python
integers, which share nothing with either side)."""
import numpy as np
import pytest

from paper_2405_14642_gb300 import workloads

BLK = 128
BIAS = np.float32(2.0 ** 23)


def _bytes(limbs):
    return np.ascontiguousarray(limbs.astype("<u4")).view(np.uint8).astype(np.int64)


def _to_int(limbs):
    return int.from_bytes(np.ascontiguousarray(limbs.astype("<u4")).tobytes(), "little")


def tc_product(a_limbs, b_limbs):
    """a * b by the block formulation; the longer operand plays X."""
    if a_limbs.size < b_limbs.size:
        a_limbs, b_limbs = b_limbs, a_limbs
    ab, bb = _bytes(a_limbs), _bytes(b_limbs)
    ma, mb = -(-ab.size // BLK), -(-bb.size // BLK)
    X = np.zeros((ma, BLK), np.int64)
    X.reshape(-1)[:ab.size] = ab
    bpad = np.zeros(BLK * (mb + 2), np.int64)  # b at offset 128, zeros around it
    bpad[BLK:BLK + bb.size] = bb
    cols = np.zeros(BLK * (ma + mb), np.int64)
    r = np.arange(BLK)[:, None]
    c = np.arange(BLK)[None, :]
    for J in range(mb + 1):
        W = bpad[BLK + BLK * J + r - c]                       # Toeplitz block of b
        s_lo, s_hi = J, J + ma                                # output blocks this J reaches
        exact = W @ X.T                                       # int64: (128, ma)
        D = BIAS + W.astype(np.float32) @ X.T.astype(np.float32)
        assert exact.max() < 2 ** 23                          # 128 * 255^2 < 2^23
        assert np.array_equal(D.astype(np.int64) - 2 ** 23, exact)
        bits = D.view(np.uint32).astype(np.int64) - 0x4B000000
        assert np.array_equal(bits, exact)                    # the bit pattern is the integer
        for I in range(ma):
            s = J + I
            cols[BLK * s:BLK * s + BLK] += bits[:, I]
        assert s_hi - s_lo == ma
    assert cols.max() < 2 ** 31
    # column sums at byte positions -> the product
    return sum(int(v) << (8 * k) for k, v in enumerate(cols))


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 5), (31, 33), (32, 32), (100, 7), (7, 100), (257, 130)])
def test_block_formulation_equals_python_product(na, nb):
    a, b = workloads.pair_batch(3, na, nb, seed=workloads.seed_for(9, 5000 + na * 3 + nb), edges=True)
    for i in range(3):
        assert tc_product(a[i], b[i]) == _to_int(a[i]) * _to_int(b[i])


def test_block_formulation_all_ones_is_the_worst_case():
    """All bytes 255: every block sum at its bound 128 * 255^2, still exact."""
    ones = np.full(64, 0xFFFFFFFF, np.uint32)
    v = (1 << (32 * 64)) - 1
    assert tc_product(ones, ones) == v * v


def test_block_size_within_the_exact_range():
    """A block's 128 byte products stay below 2^23, so on the 2^23 bias every
    partial sum is an integer in [2^23, 2^24), where f32 spacing is 1; a block
    of 130 bytes could reach 2^24, where f32 stops representing every integer."""
    assert 128 * 255 * 255 < 2 ** 23 <= 130 * 255 * 255
    assert np.float32(2.0 ** 24) + np.float32(1.0) == np.float32(2.0 ** 24)
    assert np.float32(2.0 ** 24 - 1) - np.float32(2.0 ** 23) == np.float32(2.0 ** 23 - 1)


def circular_product(a_limbs, b_limbs):
    """a * b by the circular schedule the kernel runs: D has ma columns; step
    J (0..mb) is W_J times the window of the doubled X (XX[I] = a-block I mod
    ma, zero blocks up to ma rounded to 16) that starts at block ma - J; after
    step J, column J is stored as output block J and starts over as block
    J + ma; after the last step column n goes to block n (n >= mb) or n + ma."""
    if a_limbs.size < b_limbs.size:
        a_limbs, b_limbs = b_limbs, a_limbs
    ab, bb = _bytes(a_limbs), _bytes(b_limbs)
    ma, mb = -(-ab.size // BLK), -(-bb.size // BLK)
    ma16 = -(-ma // 16) * 16
    X = np.zeros((ma, BLK), np.int64)
    X.reshape(-1)[:ab.size] = ab
    XX = np.zeros((2 * ma + ma16 - ma, BLK), np.int64)
    XX[:ma], XX[ma:2 * ma] = X, X
    bpad = np.zeros(BLK * (mb + 2), np.int64)
    bpad[BLK:BLK + bb.size] = bb
    out = np.full(BLK * (ma + mb), -1, np.int64)       # every byte column written exactly once
    acc = np.zeros((BLK, ma16), np.int64)              # the epilogue's column sums (rows r, columns n)
    r = np.arange(BLK)[:, None]
    c = np.arange(BLK)[None, :]
    for J in range(mb + 1):
        W = bpad[BLK + BLK * J + r - c]
        window = XX[ma - J:ma - J + ma16]               # the MMA's B operand: N = ma16 rows
        D = BIAS + W.astype(np.float32) @ window.T.astype(np.float32)
        acc += D.view(np.uint32).astype(np.int64) - 0x4B000000
        if J < mb:                                      # column J is complete as block J
            assert (out[BLK * J:BLK * J + BLK] == -1).all()
            out[BLK * J:BLK * J + BLK] = acc[:, J]
            acc[:, J] = 0
    for n in range(ma):
        s = n + ma if n < mb else n
        assert (out[BLK * s:BLK * s + BLK] == -1).all()
        out[BLK * s:BLK * s + BLK] = acc[:, n]
    assert (out >= 0).all() and out.max() < 2 ** 31
    return sum(int(v) << (8 * k) for k, v in enumerate(out))


@pytest.mark.parametrize("na,nb", [(1, 1), (2, 1), (33, 31), (100, 7), (7, 100), (141 * 32, 3), (300, 299)])
def test_circular_schedule_equals_python_product(na, nb):
    """Ragged block counts (ma not a multiple of 16), unequal lengths, a
    one-block operand, edge rows: the circular D gives Python's product."""
    a, b = workloads.pair_batch(3, na, nb, seed=workloads.seed_for(9, 7000 + na * 3 + nb), edges=True)
    for i in range(3):
        assert circular_product(a[i], b[i]) == _to_int(a[i]) * _to_int(b[i])


def test_circular_schedule_at_the_largest_size():
    """8192 x 8192 limbs (ma = mb = 256, the 256-column D) with all-ones
    operands, where every column sum is largest, and with random ones."""
    ones = np.full(8192, 0xFFFFFFFF, np.uint32)
    v = (1 << (32 * 8192)) - 1
    assert circular_product(ones, ones) == v * v
    a, b = workloads.pair_batch(1, 8192, 8191, seed=workloads.seed_for(9, 7777))
    assert circular_product(a[0], b[0]) == _to_int(a[0]) * _to_int(b[0])
