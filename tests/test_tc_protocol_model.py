"""The mbarrier hand-overs of the tensor-core schoolbook's 256K-bit kernel
(k_mul_quad_tc: two slots of Toeplitz rows, two D slots) and 128K-bit kernel
(k_mul_quad_tc_tw: two W slots, three D slots) checked on the CPU.

Each role is a generator of its actions in program order: ("wait", bar, k)
waits for the k-th completion of bar by its parity (mbarrier
try_wait.parity), ("arrive", bar) completes a phase (one arrival stands for
all the role's warps), ("commit", bar) queues an arrival the tensor pipe
delivers after the MMAs issued before it, ("sync", p) is the CTA-wide
barrier between products.  Random schedules must finish without a deadlock,
and every parity wait must pass exactly when completion k has happened (a
barrier two phases ahead would block it for ever, one behind would let it
through early)."""
import numpy as np
import pytest


def _run(roles, seed):
    rng = np.random.default_rng(seed)
    done, fifo = {}, []
    pending = [next(r, None) for r in roles]
    arrived = {}     # CTA barrier instance -> roles that have reached it
    waits = 0
    while True:
        ready = []
        for i, act in enumerate(pending):
            if act is not None and act[0] == "sync":
                arrived.setdefault(act[1], set()).add(i)
        for i, act in enumerate(pending):
            if act is None:
                continue
            if act[0] == "wait":
                c, k = done.get(act[1], 0), act[2]
                assert c <= k + 1, f"{act[1]} ran {c - k} phases past a wait for completion {k}"
                if c % 2 != k % 2:
                    assert c == k + 1, f"{act[1]}: wait for completion {k} passed at {c}"
                    ready.append(i)
            elif act[0] == "sync":
                if len(arrived[act[1]]) == len(roles):
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
        elif act[0] == "wait":
            waits += 1
        pending[i] = next(roles[i], None)


def _roles_256k(S, products):
    """k_mul_quad_tc: per product the CTA stages, then warp 0 issues each step
    once its T slot is built and its D slot read, warps 1-7 build each step's
    T rows once the MMAs two steps back have read the slot, warps 8-23 read
    each step's D; a CTA barrier ends the product."""
    def mma():
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for _ in range(S):
                yield ("wait", ("wfull", gs % 2), gs // 2)
                if gs >= 2:
                    yield ("wait", ("dempty", gs % 2), gs // 2 - 1)
                yield ("commit", ("dfull", gs % 2))
                yield ("commit", ("wempty", gs % 2))
                gs += 1
            yield ("sync", 2 * p + 1)

    def builders():
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for _ in range(S):
                if gs >= 2:
                    yield ("wait", ("wempty", gs % 2), gs // 2 - 1)
                yield ("arrive", ("wfull", gs % 2))
                gs += 1
            yield ("sync", 2 * p + 1)

    def epilogue():
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for _ in range(S):
                yield ("wait", ("dfull", gs % 2), gs // 2)
                yield ("arrive", ("dempty", gs % 2))
                gs += 1
            yield ("sync", 2 * p + 1)

    return [mma(), builders(), epilogue()]


def _roles_tw(S, products):
    """k_mul_quad_tc_tw: the epilogue warps build W_0, W_1, then per step wait
    for its D, build W_{J+2} into the slot step J has finished with, and free
    the D slot; warp 0 issues each step once its W is built and its D slot
    (three back) read."""
    def mma():
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for _ in range(S):
                yield ("wait", ("wfull", gs % 2), gs // 2)
                if gs >= 3:
                    yield ("wait", ("dempty", gs % 3), gs // 3 - 1)
                yield ("commit", ("dfull", gs % 3))
                gs += 1
            yield ("sync", 2 * p + 1)

    def epilogue():
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for J in range(min(2, S)):
                yield ("arrive", ("wfull", (gs + J) % 2))
            for J in range(S):
                yield ("wait", ("dfull", gs % 3), gs // 3)
                if J + 2 < S:
                    yield ("arrive", ("wfull", gs % 2))
                yield ("arrive", ("dempty", gs % 3))
                gs += 1
            yield ("sync", 2 * p + 1)

    return [mma(), epilogue()]


@pytest.mark.parametrize("S", [1, 2, 3, 4, 7, 129, 257])
@pytest.mark.parametrize("products", [1, 2, 3])
def test_256k_kernel_hand_overs(S, products):
    for seed in range(60):
        assert _run(_roles_256k(S, products), seed) > 0


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 66, 129])
@pytest.mark.parametrize("products", [1, 2, 3])
def test_tw_kernel_hand_overs(S, products):
    for seed in range(60):
        assert _run(_roles_tw(S, products), seed) > 0


def test_the_model_catches_a_missing_wait():
    """Planted in the model (not in the kernel): the 256K kernel's MMA warp
    without its wait for a read D slot lets a D barrier run ahead of the
    epilogue's waits in some schedule."""
    def mma_no_dempty(S, products):
        gs = 0
        for p in range(products):
            yield ("sync", 2 * p)
            for _ in range(S):
                yield ("wait", ("wfull", gs % 2), gs // 2)
                yield ("commit", ("dfull", gs % 2))
                yield ("commit", ("wempty", gs % 2))
                gs += 1
            yield ("sync", 2 * p + 1)
    failed = 0
    for seed in range(200):
        roles = _roles_256k(9, 2)
        roles[0] = mma_no_dempty(9, 2)
        try:
            _run(roles, seed)
        except AssertionError:
            failed += 1
    assert failed > 0
