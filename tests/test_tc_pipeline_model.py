"""The mbarrier pipelines of the tensor-core schoolbook kernels, modelled on
the CPU with the kernels' own slot and parity formulas.

Each kernel links its roles with mbarriers used as phase counters: a waiter
for phase n of a barrier tests parity n & 1, which is only sound if the
barrier never completes phase n + 1 past it (two phases ahead looks like no
phase at all: a hang).  The model runs the roles as agents under many random
interleavings, over several products per CTA (the counters run on across
products), with every MMA step completing asynchronously in issue order, and
checks: no deadlock, no parity aliasing at any wait, no W slot rewritten
before the MMAs that read it completed, no D slot reissued before the
epilogue released it.

Roles and formulas, as in the kernels:
* k_mul_quad_tc (two D slots, two W slots in shared memory): builders wait
  wempty[g % 2] for use g/2 - 1 and arrive wfull; the MMA warp waits wfull[g
  % 2] (phase g/2) and dempty[g % 2] (phase g/2 - 1), its commits arrive on
  dfull and wempty; the epilogue waits dfull[g % 2] (phase g/2) and arrives
  dempty.
* k_mul_quad_tc_tw (W in tensor memory, 128-column D slots: three D slots,
  two W slots): the epilogue builds W_0, W_1 in a prologue, then in step g's
  iteration (after dfull) builds the W of step g + 2 into slot g % 2; the MMA
  warp waits wfull (phase g/2) and dempty (phase g/3 - 1) for every step it
  issues.
The Toeplitz-window kernel (up to 64 blocks) has its own model in
tests/test_tc_tall_model.py.  run_tw also runs an earlier paired form (DW =
64: four slots of each, steps issued in pairs) that no kernel uses any more."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.completed = count, 0, 0

    def arrive(self):
        self.pending += 1
        if self.pending == self.count:
            self.pending = 0
            self.completed += 1

    def test(self, phase):
        """The hardware's parity test for `phase`, plus the aliasing check."""
        assert self.completed <= phase + 1, f"phase {phase} aliased: {self.completed} phases completed"
        return self.completed > phase


def run_tw(DW, steps_per_product, products, seed, mistake=None):
    DS, WS, pair = (3, 2, False) if DW == 128 else (4, 4, True)
    rng = random.Random(seed)
    wfull = [Barrier(1) for _ in range(WS)]  # one agent stands for the 16 epilogue warps
    dfull = [Barrier(1) for _ in range(DS)]
    dempty = [Barrier(1) for _ in range(DS)]
    issued, completed_mma = [], 0            # global steps issued to the tensor pipe, in order
    read_done = set()                        # D of global step g read by the epilogue
    w_written = {}                           # slot -> global step whose W it holds

    def mma_agent():
        gs = 0
        for S in steps_per_product:
            J = 0
            while J < S:
                n = 2 if pair and J + 1 < S else 1
                for h in range(n):
                    g = gs + h
                    while not wfull[g % WS].test(g // WS):
                        yield
                    if mistake == "skip_second_d_wait" and h == 1:
                        continue
                    if g // DS > 0:
                        target = g // DS - (0 if mistake == "d_wait_one_phase_late" else 1)
                        while not dempty[g % DS].test(target):
                            yield
                for h in range(n):
                    g = gs + h
                    assert w_written.get(g % WS) == g, "MMA reads a W slot not holding its step's W"
                    assert g < DS or (g - DS) in read_done, "D slot reissued before its read"
                    issued.append(g)
                gs += n
                J += n
                yield
            yield "product"

    def epi_agent():
        gs = 0
        for S in steps_per_product:
            for J in range(min(WS, S)):
                w_written[(gs + J) % WS] = gs + J
                wfull[(gs + J) % WS].arrive()
            for J in range(S):
                if mistake == "w_before_d_wait" and J + WS < S:
                    assert completed_mma > gs, "W slot rewritten before its MMA completed"
                while not dfull[gs % DS].test(gs // DS):
                    yield
                if J + WS < S:
                    assert completed_mma > gs, "W slot rewritten before its MMA completed"
                    w_written[gs % WS] = gs + WS
                    wfull[gs % WS].arrive()
                    yield  # the kernel releases W before it reads D
                read_done.add(gs)
                dempty[gs % DS].arrive()
                gs += 1
                yield
            yield "product"

    agents = {"mma": mma_agent(), "epi": epi_agent()}
    at_sync, done = set(), set()
    stalls = 0
    while len(done) < 2:
        choices = [a for a in agents if a not in done and a not in at_sync]
        can_complete = completed_mma < len(issued)
        if can_complete:
            choices.append("tensor")
        if not choices:  # both at the product barrier
            at_sync.clear()
            continue
        who = rng.choice(choices)
        if who == "tensor":  # the oldest issued MMA step completes: its commit arrives on dfull
            g = issued[completed_mma]
            completed_mma += 1
            dfull[g % DS].arrive()
            stalls = 0
            continue
        try:
            r = next(agents[who])
            if r == "product":
                at_sync.add(who)
        except StopIteration:
            done.add(who)
        stalls += 1
        assert stalls < 100000, "deadlock"
    assert completed_mma == len(issued) == sum(steps_per_product)


def run_smem(steps_per_product, products, seed):
    """k_mul_quad_tc: builders, MMA warp and epilogue, two slots of each."""
    rng = random.Random(seed)
    wfull = [Barrier(1) for _ in range(2)]
    wempty = [Barrier(1) for _ in range(2)]
    dfull = [Barrier(1) for _ in range(2)]
    dempty = [Barrier(1) for _ in range(2)]
    issued, completed_mma = [], 0
    w_holds, read_done = {}, set()

    def builders():
        gs = 0
        for S in steps_per_product:
            for _ in range(S):
                k, use = gs % 2, gs // 2
                if use > 0:
                    while not wempty[k].test(use - 1):
                        yield
                assert use == 0 or completed_mma > gs - 2, "W slot rewritten before its MMA completed"
                w_holds[k] = gs
                wfull[k].arrive()
                gs += 1
                yield
            yield "product"

    def mma():
        gs = 0
        for S in steps_per_product:
            for _ in range(S):
                k, d, ud = gs % 2, gs % 2, gs // 2
                while not wfull[k].test(gs // 2):
                    yield
                if ud > 0:
                    while not dempty[d].test(ud - 1):
                        yield
                assert w_holds.get(k) == gs and (gs < 2 or gs - 2 in read_done)
                issued.append(gs)
                gs += 1
                yield
            yield "product"

    def epi():
        gs = 0
        for S in steps_per_product:
            for _ in range(S):
                while not dfull[gs % 2].test(gs // 2):
                    yield
                read_done.add(gs)
                dempty[gs % 2].arrive()
                gs += 1
                yield
            yield "product"

    agents = {"b": builders(), "m": mma(), "e": epi()}
    at_sync, done, stalls = set(), set(), 0
    while len(done) < 3:
        choices = [a for a in agents if a not in done and a not in at_sync]
        if completed_mma < len(issued):
            choices.append("tensor")
        if not choices:
            at_sync.clear()
            continue
        who = rng.choice(choices)
        if who == "tensor":
            g = issued[completed_mma]
            completed_mma += 1
            dfull[g % 2].arrive()
            wempty[g % 2].arrive()
            stalls = 0
            continue
        try:
            if next(agents[who]) == "product":
                at_sync.add(who)
        except StopIteration:
            done.add(who)
        stalls += 1
        assert stalls < 100000, "deadlock"
    assert completed_mma == len(issued) == sum(steps_per_product)


# steps per product = mb + 1: 2 (one-block operand) up to odd and even counts
SHAPES = [[2, 2, 2], [3, 5, 2], [4, 4, 4, 4], [9, 2, 8, 33], [65, 64, 2]]


@pytest.mark.parametrize("steps", SHAPES, ids=lambda s: "-".join(map(str, s)))
def test_tensor_memory_w_pipeline(steps):
    for seed in range(40):
        run_tw(128, steps, len(steps), seed)


@pytest.mark.parametrize("steps", SHAPES, ids=lambda s: "-".join(map(str, s)))
def test_shared_memory_w_pipeline(steps):
    for seed in range(40):
        run_smem(steps, len(steps), seed)


@pytest.mark.parametrize("DW,mistake", [(128, "w_before_d_wait"), (128, "d_wait_one_phase_late"),
                                        (64, "skip_second_d_wait")])
def test_the_model_catches_planted_protocol_mistakes(DW, mistake):
    """Plausible slips: W rebuilt before the step that read it delivered its
    D, the D-slot wait aimed one phase late (in the protocol of the kernel),
    and, in the paired form, the second step of a pair not waiting for its D
    slot.  Each must fail (an assertion, aliasing or a deadlock) under some
    interleaving."""
    failed = False
    for seed in range(200):
        try:
            run_tw(DW, [9, 2, 8, 33], 4, seed, mistake=mistake)
        except AssertionError:
            failed = True
            break
    assert failed
