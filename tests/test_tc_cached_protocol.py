"""The hand-off protocol of the cached tensor-core apply (csrc/tc_cached.cu),
modelled on the CPU.

Six roles share rings of stages and hand work on through mbarriers waited
on by phase parity: two copiers, each as far ahead as its own ring allows
(A stage with the step record; the schedule's raw x_j loads), the MMA issuer
(one commit per row into the step-done ring; eight TMEM accumulators; MMAs
complete in issue order), the converters (raw x_j -> the schedule's slot
once every row up to LAG back has completed -- it waits for row i - LAG at
row i, so the waits of earlier rows cover the rest; one arrival of all 128
threads per row) and two epilogue groups (even and odd rows).  The schedule
is planned here by the rule the library's planner enforces (a load takes a
free slot, else the slot needed again furthest ahead among those whose last
reader is at least LAG rows back).  The model replays the kernel's per-role
waits, arrivals and commits under random interleavings, with bulk copies
landing and MMAs completing at random later times, and checks: no deadlock;
every parity wait unambiguous; an MMA reads slots that hold the x_j its
blocks need, an A stage holding its own row; no slot, raw or A stage
overwritten while a reader may still use it; the epilogue reads finished
products from an accumulator not yet reused.
"""
import random

import pytest

from test_tc_pipeline_protocol import Barrier

NS, ND, NACC, LAG, NRAW = 5, 16, 8, 2, 5
NX = ND


def plan(rows, S):
    """rows: list of column lists.  Returns per step (loads, slots) or None
    when no slot may be evicted (the library then falls back).  A load takes a
    free slot, else the slot whose x_j is needed again furthest ahead among
    those whose last reader is at least LAG rows back."""
    uses = {}
    for s, cols in enumerate(rows):
        for j in cols:
            uses.setdefault(j, []).append(s)

    def next_use(j, s):
        return next((u for u in uses[j] if u >= s), float("inf"))

    slot_of, content, last = {}, [None] * S, [-1] * S
    out = []
    for s, cols in enumerate(rows):
        loads, slots = [], []
        for j in cols:
            if j not in slot_of:
                free = [sl for sl in range(S) if content[sl] is None]
                if free:
                    sl = free[0]
                else:
                    ok = [sl for sl in range(S) if last[sl] <= s - LAG]
                    if not ok:
                        return None
                    sl = max(ok, key=lambda q: next_use(content[q], s))
                    del slot_of[content[sl]]
                content[sl] = j
                slot_of[j] = sl
                loads.append((j, sl))
            slots.append(slot_of[j])
            last[slot_of[j]] = s
        out.append((loads, slots))
    return out


def simulate(rows, S, seed, drop=None, slow_epilogue=False):
    sched = plan(rows, S)
    if sched is None:
        return False
    rnd = random.Random(seed)
    n = len(rows)
    full = [Barrier(1) for _ in range(NS)]
    done = [Barrier(1) for _ in range(ND)]
    xready = [Barrier(128) for _ in range(NX)]
    accempty = [Barrier(128) for _ in range(NACC)]
    rawfull = [Barrier(1) for _ in range(NRAW)]
    rawempty = [Barrier(128) for _ in range(NRAW)]
    astage = [None] * NS        # step whose A blocks / record a stage holds
    rawst = [None] * NRAW       # load index a raw stage holds
    slot = [None] * S           # element a slot holds
    pending = {0: [], 1: []}    # per issuer: issued rows whose MMAs have not completed, in order
    row_slots = {}              # row -> slots its MMAs read
    done_rows = set()           # rows whose MMAs completed
    copies = []                 # (kind, index, value, barrier)
    acc_owner = [None] * NACC
    epi_done = set()

    def wait(bar, phase, ring_parity=None):
        while not bar.try_wait_parity(phase & 1, phase):
            yield

    def raw_copier():
        loads = [j for i in range(n) for (j, _) in sched[i][0]]
        for nraw, j in enumerate(loads):
            q = nraw % NRAW
            if nraw >= NRAW and drop != "raw_empty":
                yield from wait(rawempty[q], nraw // NRAW - 1)
            rawfull[q].arrive_expect_tx(1)
            copies.append(("raw", q, (nraw, j), rawfull[q]))
            yield

    def copier():
        for i in range(n):
            ks = i % NS
            if i >= NS and drop != "copier_done":
                yield from wait(done[(i - NS) % ND], (i - NS) // ND)
            if i >= NS:
                assert (i - NS) in done_rows, "A stage overwritten while an MMA may read it"
            full[ks].arrive_expect_tx(1)
            copies.append(("a", ks, i, full[ks]))
            yield

    def mma():
        for i in range(n):
            ks, acc = i % NS, i % NACC
            yield from wait(xready[i % NX], i // NX)
            # no wait for the A stage: the converters waited for it before x-ready
            if i >= NACC and drop != "mma_accempty":
                yield from wait(accempty[acc], i // NACC - 1)
            assert astage[ks] == i, "MMA sees another row's A stage"
            assert acc_owner[acc] is None or acc_owner[acc] in epi_done, \
                "accumulator overwritten before its epilogue read it"
            acc_owner[acc] = i
            for j, sl in zip(rows[i], sched[i][1]):
                assert slot[sl] == j, f"row {i} reads slot {sl} holding {slot[sl]}, needs {j}"
            row_slots[i] = set(sched[i][1])
            pending[0].append(i)

    def converter():
        nraw = 0
        for i in range(n):
            ks = i % NS
            yield from wait(full[ks], i // NS)
            assert astage[ks] == i
            if i >= LAG and drop != "conv_lag":
                yield from wait(done[(i - LAG) % ND], (i - LAG) // ND)
            # the invariant the planner relies on: every row <= i - LAG has completed
            assert all(r in done_rows for r in range(max(0, i - LAG - 3), i - LAG + 1)), \
                f"row {i}'s slots written before the rows up to {i - LAG} completed"
            for (j, sl) in sched[i][0]:
                q = nraw % NRAW
                yield from wait(rawfull[q], nraw // NRAW)
                assert rawst[q] == (nraw, j), "converter reads another load's raw x"
                busy = [r for q in pending.values() for r in q if sl in row_slots[r]]
                assert not busy, f"slot {sl} overwritten while an MMA may read it"
                slot[sl] = j
                rawempty[q].arrive(128)
                nraw += 1
            xready[i % NX].arrive(128)

    def epilogue(par):
        for i in range(par, n, 2):
            acc = i % NACC
            yield from wait(done[i % ND], i // ND)
            assert i in done_rows, "epilogue before its row's MMAs completed"
            assert acc_owner[acc] == i
            epi_done.add(i)
            accempty[acc].arrive(128)

    roles = [copier(), mma(), converter(), epilogue(0), epilogue(1), raw_copier()]
    alive = [True] * 6
    for _ in range(10 ** 6):
        choices = [r for r in range(6) if alive[r]]
        if copies:
            choices.append("copy")
        for q in (0, 1):
            if pending[q]:
                choices.append(("mma", q))
        if not choices:
            break
        # slow_epilogue: the epilogue roles are picked 20 times less often, so
        # the MMAs run far ahead of them (the accumulator reuse is exercised)
        weights = [0.05 if (slow_epilogue and c in (3, 4)) else 1.0 for c in choices]
        c = rnd.choices(choices, weights)[0]
        if c == "copy":
            kind, idx, val, bar = copies.pop(rnd.randrange(len(copies)))
            if kind == "a":
                astage[idx] = val
            else:
                rawst[idx] = val
            bar.complete_tx(1)
        elif isinstance(c, tuple):
            r = pending[c[1]].pop(0)        # each issuer's MMAs complete in issue order
            done_rows.add(r)
            done[r % ND].arrive()
        else:
            try:
                next(roles[c])
            except StopIteration:
                alive[c] = False
    else:
        raise AssertionError("deadlock: roles still waiting after 10^6 steps")
    assert epi_done == set(range(n))
    return True


def strip_rows(n, L, extra=0, rnd=None):
    """Rows of an n x n periodic 5-point pattern in the kernel's strip order,
    optionally with extra random couplings (coarse-level interface rows)."""
    order = []
    for x0 in range(0, n, L):
        w = min(L, n - x0)
        for y in range(n):
            order += [x0 + i + n * y for i in range(w)]
    rows = []
    for e in order:
        x, y = e % n, e // n
        cols = sorted({e, (x + 1) % n + n * y, (x - 1) % n + n * y, x + n * ((y + 1) % n), x + n * ((y - 1) % n)})
        if extra and rnd.random() < extra:
            cols = sorted(set(cols) | {x + n * ((y + 2) % n), (x + 2) % n + n * y})
        rows.append(cols)
    return rows


@pytest.mark.parametrize("n,L,S", [(16, 4, 16), (16, 8, 33), (12, 8, 16), (8, 16, 33), (4, 4, 16), (2, 2, 8),
                                   (16, 8, 20)])
def test_strip_schedules(n, L, S):
    planned = 0
    for seed in range(40):
        rows = strip_rows(n, L)[: random.Random(seed).randint(1, n * n)]
        planned += simulate(rows, S, seed, slow_epilogue=seed % 2 == 1)
    assert planned > 0


def test_rows_with_extra_couplings_and_empty_rows():
    planned = 0
    for seed in range(60):
        rnd = random.Random(seed)
        rows = strip_rows(8, 4, extra=0.3, rnd=rnd)
        for i in rnd.sample(range(len(rows)), 3):
            rows[i] = []
        planned += simulate(rows, 33, seed)
    assert planned > 0


def test_plan_refuses_a_ring_too_small_for_the_lag():
    """Three rows of five blocks need up to 5 + 2 * 3 slots at once."""
    assert plan(strip_rows(16, 8), 6) is None
    assert plan(strip_rows(16, 8), 33) is not None


@pytest.mark.parametrize("drop", ["copier_done", "mma_accempty", "conv_lag", "raw_empty"])
def test_model_catches_a_dropped_wait(drop):
    """Leaving out any reuse wait is caught on some schedule (the checks are
    not vacuous)."""
    caught = 0
    rows = strip_rows(8, 4)
    for seed in range(150):
        try:
            simulate(rows, 10 if drop == "conv_lag" else 33, seed, drop=drop, slow_epilogue=drop == "mma_accempty")
        except AssertionError:
            caught += 1
    assert caught > 0
