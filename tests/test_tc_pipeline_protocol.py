"""The hand-off protocol of the tensor-core batched apply (csrc/tc_apply.cu),
modelled on the CPU.

The kernel's three roles -- the copier (warp 0), the MMA issuer (warp 1) and
the epilogue warps (2..5) -- share a ring of NS stages (each holding an
item's X_j hi / lo images and A_ij image) and two TMEM accumulators, and hand
work on through mbarriers that are waited on by phase parity.  This model
replays the same per-role sequence of waits, arrivals and commits (as written
in the kernel) under random interleavings, with bulk copies landing and MMAs
completing at random later times, and checks:

  * no deadlock for any row structure (empty rows, rows longer than the ring);
  * every parity wait is unambiguous: when a role waits for phase u of a
    barrier, the barrier has completed exactly u or u + 1 phases;
  * no buffer hazard: a stage is not overwritten while an MMA may still read
    it, the MMAs of an item see that item's data, an accumulator is not
    written by the next row's MMAs before its epilogue read it, an epilogue
    reads only finished products, and each non-empty row gets one epilogue.
"""
import random

import pytest


class Barrier:
    """mbarrier: expected arrival count, transaction bytes, completed phases."""

    def __init__(self, count):
        self.count, self.pending, self.tx, self.phase = count, count, 0, 0

    def arrive(self, n=1):
        self.pending -= n
        assert self.pending >= 0, "more arrivals than the phase expects"
        self._maybe_complete()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        assert self.tx >= 0
        self._maybe_complete()

    def _maybe_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait_parity(self, parity, intended_phase):
        """The hardware test (phase of this parity complete) plus the check
        that the parity names the intended phase unambiguously."""
        assert self.phase in (intended_phase, intended_phase + 1), \
            f"ambiguous parity wait: {self.phase} phases completed, waiting for phase {intended_phase}"
        return (self.phase & 1) != parity


class Ring:
    def __init__(self, n):
        self.n, self.s, self.ph = n, 0, 0

    def next(self):
        self.s += 1
        if self.s == self.n:
            self.s, self.ph = 0, self.ph ^ 1


def simulate(rows, NS, seed, drop=None):
    """drop: name of one wait to leave out (a planted mistake), or None."""
    rnd = random.Random(seed)
    full = [Barrier(1) for _ in range(NS)]
    empty = [Barrier(1) for _ in range(NS)]
    accfull = [Barrier(1) for _ in range(2)]
    accempty = [Barrier(128) for _ in range(2)]
    stage = [dict() for _ in range(NS)]      # which item's data each part of a stage holds
    issued = []            # (item, accumulator row index t) per MMA group, in issue order
    done = [0]             # MMA groups completed (in order)
    commits = []           # (groups issued when committed, barrier)
    copies = []            # bulk copies in flight: (stage, item, part)
    epilogues = set()

    def copier():
        k, r = 0, Ring(NS)
        for z in rows:
            for _ in range(z):
                if k >= NS and drop != "copier_empty":
                    while not empty[r.s].try_wait_parity(r.ph ^ 1, k // NS - 1):
                        yield
                if k >= NS:
                    assert done[0] >= k - NS + 1, "stage overwritten while an MMA may read it"
                full[r.s].arrive_expect_tx(3)
                copies.extend([(r.s, k, "xhi"), (r.s, k, "xlo"), (r.s, k, "a")])
                r.next()
                k += 1

    def mma():
        k, t, r = 0, 0, Ring(NS)
        for z in rows:
            if z == 0:
                continue
            acc = t & 1
            if t >= 2 and drop != "mma_accempty":
                while not accempty[acc].try_wait_parity(((t >> 1) - 1) & 1, (t >> 1) - 1):
                    yield
            assert t < 2 or (t - 2) in epilogues, "accumulator overwritten before its epilogue read it"
            for _ in range(z):
                while not full[r.s].try_wait_parity(r.ph, k // NS):
                    yield
                assert all(stage[r.s].get(part) == k for part in ("xhi", "xlo", "a")), \
                    f"MMA of item {k} sees another item's data"
                issued.append((k, t))
                commits.append((len(issued), empty[r.s]))
                r.next()
                k += 1
            commits.append((len(issued), accfull[acc]))
            t += 1

    def epilogue_warps():
        t = 0
        for z in rows:
            if z == 0:
                continue          # an empty row's output needs no accumulator
            acc = t & 1
            while not accfull[acc].try_wait_parity((t >> 1) & 1, t >> 1):
                yield
            assert all(issued[i][1] != t for i in range(done[0], len(issued))), "epilogue before its MMAs"
            epilogues.add(t)
            accempty[acc].arrive(128)
            t += 1

    roles = [copier(), mma(), epilogue_warps()]
    alive = [True, True, True]
    for _ in range(10 ** 6):
        choices = [i for i in range(3) if alive[i]]
        if copies:
            choices.append("copy")
        if done[0] < len(issued):
            choices.append("mma")
        if not choices:
            break
        c = rnd.choice(choices)
        if c == "copy":
            s, k, part = copies.pop(rnd.randrange(len(copies)))
            stage[s][part] = k
            full[s].complete_tx(1)
        elif c == "mma":
            done[0] += 1
            for n, bar in [cm for cm in commits if cm[0] == done[0]]:
                bar.arrive()
            commits[:] = [cm for cm in commits if cm[0] != done[0]]
        else:
            try:
                next(roles[c])
            except StopIteration:
                alive[c] = False
    else:
        raise AssertionError("deadlock: roles still waiting after 10^6 steps")
    assert len(epilogues) == sum(1 for z in rows if z)


@pytest.mark.parametrize("NS", [2, 3, 4, 6, 8])
def test_random_schedules(NS):
    for seed in range(300):
        rnd = random.Random(seed * 7 + NS)
        rows = [rnd.choice([0, 1, 1, 2, 5, 5, 5, 7, 9, 13]) for _ in range(rnd.randint(0, 14))]
        simulate(rows, NS, seed)


@pytest.mark.parametrize("drop,rows,NS", [("copier_empty", [5, 5, 5, 7, 5, 13, 5, 5], 3),
                                          ("mma_accempty", [1] * 10, 8)])
def test_model_catches_a_dropped_wait(drop, rows, NS):
    """Leaving out either reuse wait is caught by the model on some schedule
    (the checks are not vacuous).  The accumulator wait matters when the MMAs
    can run two rows ahead of the epilogue: short rows, a deep ring."""
    caught = 0
    for seed in range(200):
        try:
            simulate(rows, NS, seed, drop=drop)
        except AssertionError:
            caught += 1
    assert caught > 0
