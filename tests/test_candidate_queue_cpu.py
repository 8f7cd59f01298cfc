"""CPU model of the screen's candidate queue (k_tc_screen, csrc/screen.cu).

Epilogue warps append the pairs that pass their test to a ring of C entries
in shared memory; one candidate warp takes them.  The protocol, step by step
as the kernel takes it:

  producer lane:  t = tail; tail += 1 (the warp's lanes reserve consecutive
                  entries with one atomic); wait until t - head < C; write
                  slot t mod C; publish seq[t mod C] = t + 1.
  producer warp:  after its last entry is published, done += 1.
  consumer:       tail' = tail; if head == tail': exit once done == P and
                  tail is still head, else idle; otherwise take n =
                  min(32, tail' - head) entries: wait for each slot's
                  sequence word to read head + i + 1, read it, then head += n.

Here every step is an atomic action and a random scheduler interleaves the
producers' lanes and the consumer, with bursts that fill the ring.  Whatever
the order: every entry is taken exactly once and holds what its producer
wrote, no slot is written while an unread entry sits in it, every wait ends
(the run finishes), and the consumer leaves only after all entries are taken.
"""
import random

import pytest


class Ring:
    def __init__(self, cap):
        self.cap = cap
        self.slot = [None] * cap
        self.seq = [0] * cap
        self.tail = 0
        self.head = 0
        self.done = 0


def producer(ring, pid, items, lanes=32, wait_for_space=True):
    """One epilogue warp: groups of up to `lanes` entries reserved together;
    yields after every atomic step so the scheduler can interleave."""
    k = 0
    while k < len(items):
        group = items[k:k + random.randint(1, lanes)]
        k += len(group)
        base = ring.tail                      # one atomic add for the warp
        ring.tail += len(group)
        yield
        pending = [(base + i, v) for i, v in enumerate(group)]
        while pending:                        # lanes proceed independently
            i = random.randrange(len(pending))
            t, v = pending[i]
            if wait_for_space and t - ring.head >= ring.cap:   # no free slot yet
                yield
                continue
            s = t % ring.cap
            assert ring.seq[s] in (0, t + 1 - ring.cap) and ring.head > t - ring.cap, \
                "slot written while an unread entry sat in it"
            ring.slot[s] = (pid, v, t)
            yield
            ring.seq[s] = t + 1               # published
            pending.pop(i)
            yield
    ring.done += 1
    yield


def consumer(ring, nprod, taken):
    while True:
        tail = ring.tail
        if ring.head == tail:
            if ring.done == nprod and ring.tail == ring.head:
                return
            yield
            continue
        n = min(32, tail - ring.head)
        got = []
        for i in range(n):
            t = ring.head + i
            while ring.seq[t % ring.cap] != t + 1:
                yield
            entry = ring.slot[t % ring.cap]
            assert entry[2] == t, "read an entry other than the one published"
            got.append(entry)
        ring.head += n                        # the slots may be written again
        taken.extend(got)
        yield


@pytest.mark.parametrize("cap", [64, 256])
@pytest.mark.parametrize("seed", range(12))
def test_every_entry_taken_once_in_any_interleaving(cap, seed):
    run(cap, seed, True)


def test_the_model_catches_a_producer_that_skips_the_space_wait():
    # the same scheduler with the space wait left out overwrites unread slots
    caught = 0
    for seed in range(12):
        try:
            run(64, seed, False)
        except AssertionError:
            caught += 1
    assert caught > 0


def run(cap, seed, wait_for_space):
    random.seed(seed * 7919 + cap)
    nprod = 8
    items = {p: [random.random() for _ in range(random.choice([0, 3, 40, 300]))] for p in range(nprod)}
    ring = Ring(cap)
    taken = []
    tasks = [producer(ring, p, items[p], wait_for_space=wait_for_space) for p in range(nprod)] + \
        [consumer(ring, nprod, taken)]
    alive = list(range(len(tasks)))
    steps = 0
    while alive:
        i = random.choice(alive)
        try:
            next(tasks[i])
        except StopIteration:
            alive.remove(i)
            if i == len(tasks) - 1:            # the consumer left: every producer finished first
                assert ring.done == nprod and ring.head == ring.tail
        steps += 1
        assert steps < 2_000_000, "a wait did not end"
    expected = sorted((p, v) for p, vs in items.items() for v in vs)
    got = sorted((p, v) for p, v, _ in taken)
    assert got == expected
    assert len({t for _, _, t in taken}) == len(taken)
    assert ring.head == ring.tail == len(taken)
