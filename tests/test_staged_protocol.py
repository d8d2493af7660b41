"""CPU model of the staged step kernel's copy protocol (csrc/k_step_staged.cu).

One block: a producer copies slice s of its chunk into slot s % 4 after
every consumer has released slice s - 4 on the slot's empty barrier; each
consumer waits for the slices it reads on the slots' full barriers, updates
slice z from slices z - 1, z, z + 1, and releases slice z - 1 after it.
Barriers follow the mbarrier phase rules (a wait for parity P succeeds once
the phase with that parity has completed, and at once for the phase before
the first), copies complete after a random delay, and the threads run in a
random order.  For many chunk positions and lengths the model checks that
every thread finishes (no deadlock), that every read finds its slice landed
in its slot, and that no copy overwrites a slot a consumer may still read."""
import random

import pytest

SLOTS = 4


class Barrier:
    def __init__(self, count):
        self.count = count
        self.arrived = 0
        self.tx = 0
        self.phase = 0          # completed phases

    def _maybe_complete(self):
        if self.arrived == self.count and self.tx == 0:
            self.phase += 1
            self.arrived = 0

    def arrive(self, tx=0):
        self.tx += tx
        self.arrived += 1
        self._maybe_complete()

    def complete_tx(self, n):
        self.tx -= n
        assert self.tx >= 0
        self._maybe_complete()

    def test(self, parity):
        return (self.phase & 1) != parity


def chunk(nz, zlen, b):
    z0 = b * zlen
    z1 = min(z0 + zlen, nz)
    return z0, z1, max(z0 - 1, 0), min(z1, nz - 1)


def run_block(nz, zlen, b, consumers, rng, max_ticks=200000):
    z0, z1, lo, hi = chunk(nz, zlen, b)
    full = [Barrier(1) for _ in range(SLOTS)]
    empty = [Barrier(consumers) for _ in range(SLOTS)]
    landed = [None] * SLOTS         # slice whose copy has completed in each slot
    copies = []                     # in flight: (slot, slice, ticks left)
    progress = [None] * consumers   # iteration each consumer is in (None: prologue)

    def producer():
        for zs in range(lo, hi + 1):
            q, k = zs % SLOTS, (zs - lo) >> 2
            if k > 0:
                while not empty[q].test((k - 1) & 1):
                    yield
                # every consumer has left the last iteration that reads slice zs - 4
                for p in progress:
                    assert p is not None and p > zs - 3, (zs, progress)
            landed[q] = None
            full[q].arrive(tx=1)
            copies.append([q, zs, rng.randint(0, 6)])
            yield

    def consumer(c):
        def wait(zs):
            q = zs % SLOTS
            while not full[q].test(((zs - lo) >> 2) & 1):
                yield
            assert landed[q] == zs, (zs, q, landed[q])

        for zs in range(lo, min(z0, hi) + 1):
            yield from wait(zs)
        for z in range(z0, z1):
            progress[c] = z
            if z + 1 <= hi:
                yield from wait(z + 1)
            for s in (z - 1, z, z + 1):
                if lo <= s <= hi:
                    assert landed[s % SLOTS] == s, (z, s)
            yield
            if z - 1 >= lo:
                empty[(z - 1) % SLOTS].arrive()
            progress[c] = z + 1   # has left iteration z
        progress[c] = z1 + 10     # done

    threads = [producer()] + [consumer(c) for c in range(consumers)]
    alive = list(range(len(threads)))
    for _ in range(max_ticks):
        for cp in list(copies):
            if cp[2] == 0:
                landed[cp[0]] = cp[1]
                full[cp[0]].complete_tx(1)
                copies.remove(cp)
            else:
                cp[2] -= 1
        if not alive:
            return
        t = rng.choice(alive)
        try:
            next(threads[t])
        except StopIteration:
            alive.remove(t)
    raise AssertionError("deadlock: threads %s still waiting" % alive)


@pytest.mark.parametrize("nz,zlen", [(8, 1), (5, 1), (23, 2), (40, 3), (30, 5), (512, 27), (64, 64), (9, 4)])
def test_copy_protocol_finishes_and_reads_landed_slices(nz, zlen):
    rng = random.Random(1000 * nz + zlen)
    nblocks = (nz + zlen - 1) // zlen
    for b in range(nblocks):
        for consumers in (1, 3, 5):
            run_block(nz, zlen, b, consumers, rng)


def test_model_catches_a_release_that_comes_one_iteration_early():
    """The model is not vacuous: releasing slice z - 1 before the update of
    slice z (instead of after it) lets a copy overwrite a slot that is still
    read, which the model reports."""
    rng = random.Random(3)

    def early(nz, zlen, b, consumers):
        z0, z1, lo, hi = chunk(nz, zlen, b)
        full = [Barrier(1) for _ in range(SLOTS)]
        empty = [Barrier(consumers) for _ in range(SLOTS)]
        landed = [None] * SLOTS
        copies = []
        bad = []

        def producer():
            for zs in range(lo, hi + 1):
                q, k = zs % SLOTS, (zs - lo) >> 2
                if k > 0:
                    while not empty[q].test((k - 1) & 1):
                        yield
                landed[q] = None
                full[q].arrive(tx=1)
                copies.append([q, zs, rng.randint(0, 6)])
                yield

        def consumer(c):
            for zs in range(lo, min(z0, hi) + 1):
                while not full[zs % SLOTS].test(((zs - lo) >> 2) & 1):
                    yield
            for z in range(z0, z1):
                if z + 1 <= hi:
                    while not full[(z + 1) % SLOTS].test(((z + 1 - lo) >> 2) & 1):
                        yield
                if z - 1 >= lo:
                    empty[(z - 1) % SLOTS].arrive()   # too early
                for _ in range(3):
                    yield
                for s in (z - 1, z, z + 1):
                    if lo <= s <= hi and landed[s % SLOTS] != s:
                        bad.append((z, s))

        threads = [producer()] + [consumer(c) for c in range(consumers)]
        alive = list(range(len(threads)))
        while alive:
            for cp in list(copies):
                if cp[2] == 0:
                    landed[cp[0]] = cp[1]
                    full[cp[0]].complete_tx(1)
                    copies.remove(cp)
                else:
                    cp[2] -= 1
            t = rng.choice(alive)
            try:
                next(threads[t])
            except StopIteration:
                alive.remove(t)
        return bad

    found = []
    for trial in range(40):
        found += early(60, 30, 1, 2)
    assert found
