"""A model of the barrier protocol of the fused MLP forward kernel
(k_mlp_fused: one persistent CTA per SM, two 128-row tiles in flight), run
on the CPU under random interleavings of its three roles and of the
asynchronous completions (TMA copies in any order, tensor-core commits in
issue order).  It checks that no wait deadlocks, that no mbarrier completes
two phases past the phase its waiter expects (a parity wait would then
miss it), and that every buffer and accumulator is read only after it holds
the data the step needs and overwritten only after its last reader is done.
Planted mistakes in the model (a missing wait, one barrier shared by both
slots) must be caught.

The model follows the kernel's work-item order: for each pair of tiles,
layer 0..3, slot 0 then slot 1.  Per slot: x_full (input tile landed),
buf_free (the slot's last-layer MMAs done), acc_full (the slot's
accumulator complete), epi_done (the epilogue of the slot's layer done);
per ring stage: full, empty."""
import random

import pytest

KB_IN, KB_H, STAGES = 5, 4, 2


class _Bar:
    def __init__(self, count=1):
        self.count, self.pending, self.phase = count, 0, 0

    def arrive(self):
        self.pending += 1
        if self.pending == self.count:
            self.pending = 0
            self.phase += 1


def _run(ntl, seed, mutate=None):
    rnd = random.Random(seed)
    mutate = mutate or set()
    items = 8 * ((ntl + 1) // 2)
    bars = {}
    for s in range(STAGES):
        bars["full", s] = _Bar()
        bars["empty", s] = _Bar()
    for j in range(2):
        for n in ("x_full", "buf_free", "acc_full", "epi_done"):
            bars[n, j] = _Bar()
    if "shared_acc_barrier" in mutate:
        bars["acc_full", 1] = bars["acc_full", 0]
    pending = []  # ("t" | "m", action): TMA completions, tensor-core completions
    buf = [None, None]           # what the slot's buffer holds
    acc = [None, None]           # what the slot's accumulator holds
    mma_reading = [0, 0]         # MMAs in flight on the slot's buffer

    def wait(key, parity, expected):
        b = bars[key]
        assert b.phase <= expected + 1, ("ran ahead", key, b.phase, expected)
        while (b.phase & 1) == parity:
            yield
            assert b.phase <= expected + 1, ("ran ahead", key, b.phase, expected)

    def decode(it):
        p, l, j = it >> 3, (it >> 1) & 3, it & 1
        return p, l, j, 2 * p + j

    def loader():
        g = 0
        for it in range(items):
            p, l, j, i = decode(it)
            if i >= ntl:
                continue
            if l == 0:
                if p > 0 and "no_buf_free_wait" not in mutate:
                    yield from wait(("buf_free", j), (p - 1) & 1, p - 1)

                def land(j=j, i=i):
                    assert mma_reading[j] == 0, "input tile lands on a buffer the MMAs read"
                    buf[j] = ("x", i)
                    bars["x_full", j].arrive()
                pending.append(("t", land))
            for _ in range(KB_IN if l == 0 else KB_H):
                s = g % STAGES
                if g >= STAGES:
                    yield from wait(("empty", s), (g // STAGES - 1) & 1, g // STAGES - 1)
                pending.append(("t", lambda s=s: bars["full", s].arrive()))
                g += 1
                yield

    def mma():
        g = 0
        for it in range(items):
            p, l, j, i = decode(it)
            if i >= ntl:
                continue
            if l == 0:
                yield from wait(("x_full", j), p & 1, p)
                if p > 0 and "no_epi_wait_layer0" not in mutate:
                    yield from wait(("epi_done", j), 1, 4 * (p - 1) + 3)
            else:
                yield from wait(("epi_done", j), (l - 1) & 1, 4 * p + l - 1)
            want = ("x", i) if l == 0 else ("h", i, l - 1)
            assert buf[j] == want, ("MMA input", buf[j], want)
            free = None if (l == 0 and p == 0) else (("read", i - 2, 3) if l == 0 else ("read", i, l - 1))
            assert acc[j] == free, ("accumulator still in use", acc[j], i, l)
            mma_reading[j] += 1
            for _ in range(KB_IN if l == 0 else KB_H):
                s = g % STAGES
                yield from wait(("full", s), (g // STAGES) & 1, g // STAGES)
                pending.append(("m", lambda s=s: bars["empty", s].arrive()))
                g += 1
                yield

            def done(j=j, i=i, l=l):
                mma_reading[j] -= 1
                acc[j] = ("full", i, l)
                if l == 3:
                    bars["buf_free", j].arrive()
                bars["acc_full", j].arrive()
            pending.append(("m", done))

    def epilogue():
        for it in range(items):
            p, l, j, i = decode(it)
            if i >= ntl:
                continue
            yield from wait(("acc_full", j), l & 1, 4 * p + l)
            assert acc[j] == ("full", i, l), ("epilogue reads", acc[j], i, l)
            assert mma_reading[j] == 0, "epilogue writes a buffer the MMAs read"
            yield
            if l < 3:
                buf[j] = ("h", i, l)
            acc[j] = ("read", i, l)
            bars["epi_done", j].arrive()

    roles = {"load": loader(), "mma": mma(), "epilogue": epilogue()}
    # every run draws its own relative speeds, so that each role is, in
    # some runs, far ahead of or far behind the others
    speed = {name: rnd.choice([0.02, 0.2, 1.0, 5.0]) for name in roles}
    p_complete = rnd.choice([0.05, 0.3, 0.8])
    steps = 0
    while roles or pending:
        steps += 1
        assert steps < 200000, ("deadlock", sorted(roles))
        if pending and (not roles or rnd.random() < p_complete):
            k = rnd.randrange(len(pending))
            if pending[k][0] == "m":  # tensor-core work completes in issue order
                k = next(x for x in range(len(pending)) if pending[x][0] == "m")
            pending.pop(k)[1]()
            continue
        names = sorted(roles)
        name = rnd.choices(names, weights=[speed[n] for n in names])[0]
        try:
            next(roles[name])
        except StopIteration:
            del roles[name]


@pytest.mark.parametrize("ntl", [1, 2, 3, 4, 5])
def test_protocol_holds_under_random_interleavings(ntl):
    for seed in range(150):
        _run(ntl, seed)


@pytest.mark.parametrize("mistake", ["no_epi_wait_layer0", "shared_acc_barrier"])
def test_planted_mistakes_are_caught(mistake):
    with pytest.raises(AssertionError):
        for seed in range(150):
            for ntl in (2, 3, 4):
                _run(ntl, seed, {mistake})


def test_buffer_free_is_implied_by_the_weight_ring():
    """Without the buf_free wait the protocol still holds: the loader issues
    the next input tile only after the ring stages of the slot's last layer
    were released, and tensor-core completions are in issue order.  The
    barrier stays in the kernel as a direct statement of the dependency."""
    for seed in range(150):
        for ntl in (2, 3, 4):
            _run(ntl, seed, {"no_buf_free_wait"})
