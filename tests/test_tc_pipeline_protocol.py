"""The hand-off protocol of the tensor-core batched apply (csrc/tc_apply.cu),
modelled on the CPU.

The kernel's three roles -- the copier (warp 0), the MMA issuer (warp 1) and
the converter / epilogue warps (2..5) -- share a ring of NR raw stages, a ring
of NO operand stages and two TMEM accumulators, and hand work on through
mbarriers that are waited on by phase parity.  This model replays the same
per-role sequence of waits, arrivals and commits (as written in the kernel)
under random interleavings, with bulk copies landing and MMAs completing at
random later times, and checks:

  * no deadlock for any row structure (empty rows, rows longer than a ring);
  * every parity wait is unambiguous: when a role waits for phase u of a
    barrier, the barrier has completed exactly u or u + 1 phases;
  * no buffer hazard: a raw stage is not overwritten while an MMA may still
    read its A image, an operand stage is not rewritten while its MMA runs,
    an accumulator is not reused before its epilogue read it, the MMAs of an
    item see the data of that item, and each non-empty row gets one epilogue.
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


def simulate(rows, NR, NO, seed, drop=None):
    """drop: name of one wait to leave out (a planted mistake), or None."""
    rnd = random.Random(seed)
    rfull = [Barrier(1) for _ in range(NR)]
    rempty = [Barrier(1) for _ in range(NR)]
    ofull = [Barrier(128) for _ in range(NO)]
    oempty = [Barrier(1) for _ in range(NO)]
    accfull = [Barrier(1) for _ in range(2)]
    accempty = [Barrier(128) for _ in range(2)]
    raw_x, raw_a, opx = [None] * NR, [None] * NR, [None] * NO
    issued = []            # (item, accumulator row index t) per MMA group, in issue order
    done = [0]             # MMA groups completed (in order)
    commits = []           # (groups issued when committed, barrier)
    copies = []            # bulk copies in flight: (stage, item, which)
    epilogues = set()

    def copier():
        k, r = 0, Ring(NR)
        for z in rows:
            for _ in range(z):
                if k >= NR and drop != "copier_rempty":
                    while not rempty[r.s].try_wait_parity(r.ph ^ 1, k // NR - 1):
                        yield
                if k >= NR:
                    assert done[0] >= k - NR + 1, "raw stage overwritten while an MMA may read it"
                rfull[r.s].arrive_expect_tx(2)
                copies.extend([(r.s, k, "x"), (r.s, k, "a")])
                r.next()
                k += 1

    def mma():
        k, t, r, o = 0, 0, Ring(NR), Ring(NO)
        for z in rows:
            if z == 0:
                continue
            acc = t & 1
            if t >= 2 and drop != "mma_accempty":
                while not accempty[acc].try_wait_parity(((t >> 1) - 1) & 1, (t >> 1) - 1):
                    yield
            assert t < 2 or (t - 2) in epilogues, "accumulator reused before its epilogue"
            for _ in range(z):
                while not rfull[r.s].try_wait_parity(r.ph, k // NR):
                    yield
                while not ofull[o.s].try_wait_parity(o.ph, k // NO):
                    yield
                assert raw_a[r.s] == k and opx[o.s] == k, f"MMA of item {k} sees another item's data"
                issued.append((k, t))
                commits.extend([(len(issued), rempty[r.s]), (len(issued), oempty[o.s])])
                r.next()
                o.next()
                k += 1
            commits.append((len(issued), accfull[acc]))
            t += 1

    def converters():
        k, t, prev, r, o = 0, 0, None, Ring(NR), Ring(NO)

        def epilogue(tr):
            acc = tr & 1
            while not accfull[acc].try_wait_parity((tr >> 1) & 1, tr >> 1):
                yield
            assert all(issued[i][1] != tr for i in range(done[0], len(issued))), "epilogue before its MMAs"
            epilogues.add(tr)
            accempty[acc].arrive(128)

        for z in rows:
            for _ in range(z):
                while not rfull[r.s].try_wait_parity(r.ph, k // NR):
                    yield
                if k >= NO and drop != "converter_oempty":
                    while not oempty[o.s].try_wait_parity(o.ph ^ 1, k // NO - 1):
                        yield
                if k >= NO:
                    assert done[0] >= k - NO + 1, "operand stage rewritten while its MMA runs"
                assert raw_x[r.s] == k
                opx[o.s] = k
                ofull[o.s].arrive(128)
                r.next()
                o.next()
                k += 1
            if prev is not None:
                yield from epilogue(prev)
                prev = None
            if z:
                prev, t = t, t + 1
        if prev is not None:
            yield from epilogue(prev)

    roles = [copier(), mma(), converters()]
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
            s, k, which = copies.pop(rnd.randrange(len(copies)))
            (raw_x if which == "x" else raw_a)[s] = k
            rfull[s].complete_tx(1)
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


@pytest.mark.parametrize("NR,NO", [(2, 2), (3, 3), (6, 3), (8, 2), (4, 4)])
def test_random_schedules(NR, NO):
    for seed in range(300):
        rnd = random.Random(seed * 7 + NR)
        rows = [rnd.choice([0, 1, 1, 2, 5, 5, 5, 7, 9, 13]) for _ in range(rnd.randint(0, 14))]
        simulate(rows, NR, NO, seed)


@pytest.mark.parametrize("drop", ["copier_rempty", "converter_oempty"])
def test_model_catches_a_dropped_wait(drop):
    """Leaving out either stage-reuse wait is caught by the model on some
    schedule (the checks are not vacuous)."""
    caught = 0
    for seed in range(200):
        try:
            simulate([5, 5, 5, 7, 5, 13, 5, 5], 3, 2, seed, drop=drop)
        except AssertionError:
            caught += 1
    assert caught > 0


def test_accumulator_wait_is_implied_by_the_converter_order():
    """The MMA issuer's wait for an accumulator's epilogue never blocks in the
    model: the converters read the accumulator of row t - 2 before they
    convert row t, and the MMAs of row t need those conversions.  The kernel
    keeps the wait all the same, for the tcgen05 ordering of the TMEM read
    (tcgen05.ld, then fence::before_thread_sync and the arrival) against the
    next MMA's write."""
    for seed in range(200):
        simulate([5, 5, 5, 7, 5, 13, 5, 5], 3, 2, seed, drop="mma_accempty")
