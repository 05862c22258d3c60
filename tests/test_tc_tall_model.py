"""CPU model of the tensor-core schoolbook's form up to 64K bits, where every
MMA's A operand is a 128-row window of one tall Toeplitz matrix
T[R][c] = b-byte (R - c), c < 16, kept in shared memory (Section 3, Eq. 1's
column sums on bytes).

It checks the indexing the kernel relies on, not the oracle: K-chunk kk of
W_J (W_J[r][c] = b-byte (128 J + r - c)) equals rows R0 = 128 J - 16 kk ..
R0 + 127 of T for every step of every chunk, from the chunk's first stored
row 128 J0 - 112; the row builder's byte selection (five words of b's bytes,
byte_perm with the kernel's selector) yields exactly b-bytes R, R-1, ..., R-15
in its eight fp16 pairs without reading outside the staged words; and the
double-buffered shared-memory layout stays inside the 227 KB a CTA may hold.
A planted slip (the window one K-chunk off, the selector one byte off)
must fail."""
import numpy as np
import pytest

BLK, LEAD, ROWB = 128, 112, 32
SMEM_MAX = 227 * 1024


def byte_perm(x, y, s):
    v = (y << 32) | x
    return sum(((v >> (8 * ((s >> (4 * i)) & 7))) & 0xFF) << (8 * i) for i in range(4))


def staged_b(bbytes, mb):
    """braw: b's bytes at byte offset 128, zeros around, 32 (mb + 2) + 4 words."""
    words = 32 * (mb + 2) + 4
    raw = np.zeros(4 * words, np.int64)
    raw[128:128 + bbytes.size] = bbytes
    w = [int(raw[4 * i]) | int(raw[4 * i + 1]) << 8 | int(raw[4 * i + 2]) << 16 | int(raw[4 * i + 3]) << 24
         for i in range(words)]
    return w


def tall_row(braw, R, slip=0):
    """The kernel's row builder: returns the 16 bytes (c = 0..15) it converts."""
    e = 113 + R
    assert e >= 0
    w0, sh = e >> 2, e & 3
    assert w0 + 4 < len(braw), "reads past the staged words"
    wv = braw[w0:w0 + 5]
    sel = (sh + 3 + slip) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12)
    out = []
    for m in range(4):
        x = byte_perm(wv[3 - m], wv[4 - m], sel)
        out += [x & 0xFF, (x >> 8) & 0xFF, (x >> 16) & 0xFF, (x >> 24) & 0xFF]
    return out


def chunk_of(mb, ma16, na_limbs, nb_limbs):
    """Steps per T buffer (one group: half the D slots) and the end of the
    shared-memory layout, as the kernel's geometry lays them out."""
    ma = -(-na_limbs // 32)
    xs = (2 * ma + (ma16 - ma)) * 16
    nout = na_limbs + nb_limbs
    dw = 32 if ma16 <= 32 else 64
    group = 512 // dw // 2
    xbytes = (16 * xs + 1023) & ~1023
    t_bytes = ((BLK * group + LEAD) * ROWB + 1023) & ~1023
    off = 2 * xbytes + 3 * t_bytes                     # three T buffers
    off += ((4 * (nout + (nout >> 4)) + 16 + 15) & ~15) + 8 * 256
    off += 128 * ma                                    # a's words of the next product
    off += 2 * 4 * (32 * (mb + 2) + 4)
    off = (off + 15) & ~15
    off += 4 * 16
    off = (off + 15) & ~15
    end = off + 8 * (2 * 3 + 12) + 16                  # 18 mbarriers, the slot, the abort flag
    assert (BLK * group + LEAD) * ROWB <= t_bytes
    return group, end


@pytest.mark.parametrize("nb_limbs", [1, 31, 32, 33, 1000, 1024, 2048])
def test_windows_of_T_are_the_K_chunks_of_W(nb_limbs):
    rng = np.random.default_rng(nb_limbs)
    bb = rng.integers(0, 256, 4 * nb_limbs)
    mb = -(-bb.size // BLK)
    bpad = np.zeros(BLK * (mb + 3), np.int64)
    bpad[BLK:BLK + bb.size] = bb                       # b-byte i at BLK + i
    na_limbs = max(nb_limbs, 1024 if nb_limbs <= 1024 else 2048)
    ma16 = (-(-na_limbs // 32) + 15) & ~15
    chunk, end = chunk_of(mb, ma16, na_limbs, nb_limbs)
    assert end <= SMEM_MAX
    braw = staged_b(bb, mb)
    r = np.arange(BLK)[:, None]
    c = np.arange(16)[None, :]
    for J0 in range(0, mb + 1, chunk):
        J1 = min(mb + 1, J0 + chunk)
        Rbase, nrows = BLK * J0 - LEAD, BLK * (J1 - J0) + LEAD
        T = np.array([tall_row(braw, Rbase + i) for i in range(nrows)])
        Rs = Rbase + np.arange(nrows)[:, None]
        assert np.array_equal(T, bpad[BLK + Rs - c] * ((Rs - c) >= 0))
        for J in range(J0, J1):
            for kk in range(8):
                i0 = BLK * (J - J0) + LEAD - 16 * kk
                assert 0 <= i0 and i0 + BLK <= nrows and i0 % 8 == 0
                W_chunk = bpad[BLK + BLK * J + r - 16 * kk - c]
                assert np.array_equal(T[i0:i0 + BLK], W_chunk)


def test_planted_slips_fail():
    bb = np.random.default_rng(1).integers(1, 256, 4 * 64)
    mb = 2
    braw = staged_b(bb, mb)
    bpad = np.zeros(BLK * (mb + 3), np.int64)
    bpad[BLK:BLK + bb.size] = bb
    R = 200
    want = [int(bpad[BLK + R - cc]) for cc in range(16)]
    assert tall_row(braw, R) == want
    assert tall_row(braw, R, slip=1) != want
    # a window one K-chunk off is another matrix
    T = np.array([tall_row(braw, -LEAD + i) for i in range(BLK * 3 + LEAD)])
    r = np.arange(BLK)[:, None]
    c = np.arange(16)[None, :]
    J, kk = 1, 3
    i0 = BLK * J + LEAD - 16 * (kk + 1)
    assert not np.array_equal(T[i0:i0 + BLK], bpad[BLK + BLK * J + r - 16 * kk - c])


@pytest.mark.parametrize("limbs", [32 * k for k in range(1, 65)])
def test_layout_fits_at_every_size(limbs):
    ma = mb = -(-limbs // 32)
    ma16 = (ma + 15) & ~15
    chunk, end = chunk_of(mb, ma16, limbs, limbs)
    assert chunk >= 1 and end <= SMEM_MAX


@pytest.mark.parametrize("nb_limbs", [4097, 6000, 8192])
def test_per_step_slots_of_the_256K_kernel(nb_limbs):
    """The 256K-bit kernel builds T's 240 rows of one step at a time (rows
    128 J - 112 .. 128 J + 127): its eight K-chunk windows are W_J's, and the
    row builder stays inside the staged bytes up to the last step."""
    rng = np.random.default_rng(nb_limbs)
    bb = rng.integers(0, 256, 4 * nb_limbs)
    mb = -(-bb.size // BLK)
    bpad = np.zeros(BLK * (mb + 3), np.int64)
    bpad[BLK:BLK + bb.size] = bb
    braw = staged_b(bb, mb)
    r = np.arange(BLK)[:, None]
    c = np.arange(16)[None, :]
    for J in (0, 1, mb // 2, mb - 1, mb):
        T = np.array([tall_row(braw, BLK * J - LEAD + i) for i in range(BLK + LEAD)])
        for kk in range(8):
            i0 = LEAD - 16 * kk
            assert np.array_equal(T[i0:i0 + BLK], bpad[BLK + BLK * J + r - 16 * kk - c])


# ---- the Toeplitz-window kernel's hand-over protocol --------------------------
#
# The roles of k_mul_quad_tc_tall in program order, as generators of actions on
# mbarriers: ("wait", bar, k) waits for the k-th completion of bar with the parity
# k % 2 (mbarrier try_wait.parity), ("arrive", bar) completes a phase (each role
# stands for all its warps), ("commit", bar) queues an arrival that the tensor
# pipe delivers after every MMA issued before it.  A random scheduler runs them;
# a parity wait is only correct if, when its parity test passes, exactly k + 1
# phases have completed (a barrier two phases ahead would make it wait forever,
# one behind would let it through early).

def _tall_roles(S, kC, products, normalizer):
    groups = [min(kC, S - J) for J in range(0, S, kC)]

    def mma():
        gg = 0
        for pi in range(products):
            yield ("wait", ("xfull", pi % 2), pi // 2)
            for k, n in enumerate(groups):
                if gg >= 2:
                    yield ("wait", ("dempty", gg % 2), (gg - 2) // 2)
                yield ("wait", ("tfull", gg % 3), gg // 3)
                yield ("commit", ("tempty", gg % 3))
                if k == len(groups) - 1:
                    yield ("commit", ("xempty", pi % 2))
                gg += 1
        if gg:
            yield ("wait", ("tempty", (gg - 1) % 3), (gg - 1) // 3)

    def epilogue():
        eg = 0
        for pi in range(products):
            if pi >= 2:
                yield ("wait", ("cempty", pi % 2), (pi - 2) // 2)
            for n in groups:
                yield ("wait", ("tempty", eg % 3), eg // 3)
                yield ("arrive", ("dempty", eg % 2))
                eg += 1
            yield ("arrive", ("cfull", pi % 2))

    def finish(q):
        yield ("wait", ("cfull", q % 2), q // 2)
        yield ("arrive", ("cempty", q % 2))

    def producer():
        gg = 0
        for pi in range(products):
            if pi >= 2:
                yield ("wait", ("xempty", pi % 2), (pi - 2) // 2)
            yield ("arrive", ("xfull", pi % 2))
            for k, n in enumerate(groups):
                if gg >= 3:
                    yield ("wait", ("tempty", gg % 3), (gg - 3) // 3)
                yield ("arrive", ("tfull", gg % 3))
                last = k == len(groups) - 1
                if not normalizer and pi > 0 and (k == 2 or (last and k < 2)):
                    yield from finish(pi - 1)
                gg += 1
        if not normalizer and products:
            yield from finish(products - 1)

    def normalizing():
        for pi in range(products):
            yield from finish(pi)

    roles = [mma(), epilogue(), producer()]
    if normalizer:
        roles.append(normalizing())
    return roles


def _run_protocol(S, kC, products, normalizer, seed):
    rng = np.random.default_rng(seed)
    done = {}        # completed phases per barrier
    fifo = []        # commits the tensor pipe has yet to deliver
    roles = _tall_roles(S, kC, products, normalizer)
    pending = [next(r, None) for r in roles]
    waits = 0
    while True:
        ready = []
        for i, act in enumerate(pending):
            if act is None:
                continue
            if act[0] == "wait":
                c, k = done.get(act[1], 0), act[2]
                assert c <= k + 1, f"{act[1]} ran {c - k} phases past a wait for completion {k}"
                if c % 2 != k % 2:           # the parity test passes ...
                    assert c == k + 1, f"{act[1]}: wait for completion {k} passed at {c}"
                    ready.append(i)
            else:
                ready.append(i)
        if fifo:
            ready.append(-1)
        if not ready:
            assert all(a is None for a in pending), f"deadlock: {pending}"
            return waits
        i = ready[rng.integers(len(ready))]
        if i == -1:
            bar = fifo.pop(0)
            done[bar] = done.get(bar, 0) + 1
            continue
        act = pending[i]
        if act[0] == "arrive":
            done[act[1]] = done.get(act[1], 0) + 1
        elif act[0] == "commit":
            fifo.append(act[1])
        else:
            waits += 1
        pending[i] = next(roles[i], None)


@pytest.mark.parametrize("S,kC,normalizer", [(17, 8, False), (33, 8, False), (9, 8, False), (2, 8, False),
                                             (65, 4, True), (33, 4, True), (5, 4, True), (1, 4, True)])
@pytest.mark.parametrize("products", [1, 2, 3, 5])
def test_hand_over_protocol_under_random_schedules(S, kC, normalizer, products):
    """Steps per product S (tail groups included), 8 steps per group with the
    producer carrying the limbs (32-column slots) or 4 with four normalising
    warps (64-column slots), 1-5 products per CTA: in 150 random interleavings
    every wait completes on its own phase and no role is left waiting."""
    for seed in range(150):
        assert _run_protocol(S, kC, products, normalizer, seed) > 0
