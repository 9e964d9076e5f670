"""Step-level models of the commit protocols of OCC, NO_WAIT 2PL, 2PL
wait-die, basic TO and TicToc (CPU only).

Each transaction is a sequence of atomic shared-memory steps -- the loads,
CASes, atomics and stores of the execute kernel's attempt, in the kernel's
order -- and a seeded random scheduler interleaves the transactions of a
small scenario.  For every schedule, the transactions that committed,
replayed one after another in their reported commit order from the initial
state, must reproduce every value they read and the final state: the
definition of serializability the CUDA path is tested against, applied to the
protocol itself.  Variants that were considered and rejected are modelled as
negative controls, and the check must find a counterexample for each: OCC
with the commit timestamp taken together with (not after) the write locks,
2PL with the ticket taken before the lock point, basic TO reading without
checking wts again after the value, and TicToc reading (wts, value, rts)
without re-checking wts.  The same check covers the orders in which writers
read a record's value (TO: between the word and the dirty mark; multi-version
TO: the slot's newest version between the head and the pending mark) with
the read placed before the word or head as the negative control, and OCC's
group commit (a unit of members committed in one tenure of their shared
record) with the in-unit composition dropped as the negative control.
"""
import random
import sys

import pytest

LOCK = 1 << 62


class Mem:
    """Per-record shared state: value, a control word and (TicToc) an rts."""

    def __init__(self, values):
        self.val = list(values)
        self.word = [0] * len(values)      # OCC: version | LOCK;  TicToc: wts | LOCK
        self.rts = [0] * len(values)       # TicToc only
        self.clock = 0                     # OCC commit timestamps
        self.seq = 0                       # TicToc sequence numbers


# ---------------------------------------------------------------------------
# OCC: read phase, lock write set (no wait), timestamp, validate, write,
# publish version = timestamp + 1.  Each `yield` ends one atomic step.
# ---------------------------------------------------------------------------
def occ_txn(m, ops, out, ticket_with_locks=False):
    obs, reads, newv = {}, {}, {}
    for (r, d) in ops:                                  # read phase
        v1 = m.word[r]
        yield
        if v1 & LOCK:
            return
        x = m.val[r]
        yield
        obs[r], reads[r] = v1, x
        if d is not None:
            newv[r] = x + d
    held = []
    ts = None
    if ticket_with_locks:                               # rejected variant
        ts = m.clock
        m.clock += 1
        yield
    for (r, d) in ops:                                  # lock the write set
        if d is None:
            continue
        if m.word[r] != obs[r]:
            for h in held:
                m.word[h] = obs[h]
            return
        m.word[r] = obs[r] | LOCK
        held.append(r)
        yield
    if ts is None:                                      # the design: after the locks
        ts = m.clock
        m.clock += 1
        yield
    for (r, d) in ops:                                  # validate the read set
        if d is None:
            ok = m.word[r] == obs[r]
            yield
            if not ok:
                for h in held:
                    m.word[h] = obs[h]
                return
    for r in held:                                      # write, then publish
        m.val[r] = newv[r]
        yield
    for r in held:
        m.word[r] = ts + 1
        yield
    out.append(((ts,), reads))


# ---------------------------------------------------------------------------
# TicToc: read (wts, value, rts) as a snapshot, lock writes by a CAS that
# fixes the rts, timestamp = max(wts of reads, locked rts + 1 of writes),
# sequence number, extend rts of reads not covered, write, publish [ts, ts].
# ---------------------------------------------------------------------------
def tictoc_txn(m, ops, out, recheck=True):
    obs, rts_obs, reads, newv = {}, {}, {}, {}
    for (r, d) in ops:                                  # read phase
        y1 = m.word[r]
        yield
        if y1 & LOCK:
            return
        x = m.val[r]
        yield
        rt = m.rts[r]
        yield
        if recheck:
            y2 = m.word[r]
            yield
            if y2 != y1:
                return
        obs[r], rts_obs[r], reads[r] = y1, rt, x
        if d is not None:
            newv[r] = x + d
    held = []
    for (r, d) in ops:                                  # lock the write set
        if d is None:
            continue
        while True:                                     # 128-bit CAS on (rts, wts)
            cur_w, cur_r = m.word[r], m.rts[r]
            if cur_w == obs[r] and cur_r == rts_obs[r]:
                m.word[r] = obs[r] | LOCK
                yield
                break
            yield
            if cur_w != obs[r]:
                for h in held:
                    m.word[h] = obs[h]
                return
            rts_obs[r] = cur_r                          # only rts moved: lock at it
        held.append(r)
    ts = 0
    for (r, d) in ops:
        ts = max(ts, rts_obs[r] + 1 if d is not None else obs[r])
    sq = m.seq                                          # sequence number
    m.seq += 1
    yield
    for (r, d) in ops:                                  # validate / extend reads
        if d is not None or rts_obs[r] >= ts:
            continue
        while True:
            cur_w, cur_r = m.word[r], m.rts[r]
            yield
            if cur_w != obs[r]:
                for h in held:
                    m.word[h] = obs[h]
                return
            if cur_r >= ts:
                break
            if m.word[r] == cur_w and m.rts[r] == cur_r:    # the CAS
                m.rts[r] = ts
                yield
                break
    for r in held:                                      # write, publish [ts, ts]
        m.val[r] = newv[r]
        yield
        m.rts[r] = ts
        yield
        m.word[r] = ts
        yield
    out.append(((ts, sq), reads))


# ---------------------------------------------------------------------------
# 2PL: shared / exclusive lock words (NO_WAIT dies at once; wait-die lets an
# older requester wait, a bounded number of steps, for a younger exclusive
# holder), values read under the locks, the commit ticket taken while every
# lock is held, writes, releases.
# ---------------------------------------------------------------------------
X = 1 << 40
WAIT_STEPS = 6


def tpl_txn(m, ops, out, tid, wait_die=False, ticket_first=False):
    reads, newv, held = {}, {}, []
    ts = None
    if ticket_first:                                    # rejected variant
        ts = m.clock
        m.clock += 1
        yield
    fail = False
    for (r, d) in ops:
        waited = 0
        while True:
            w = m.word[r]
            if d is None and not (w & X):
                m.word[r] = w + 1                       # CAS w -> w + one share
                break
            if d is not None and w == 0:
                m.word[r] = X | (tid + 1)               # CAS 0 -> exclusive
                break
            yield
            if wait_die and (w & X) and tid + 1 < (w & (X - 1)) and waited < WAIT_STEPS:
                waited += 1                             # older: wait for the younger holder
                continue
            fail = True
            break
        if fail:
            break
        held.append((r, d))
        yield
        x = m.val[r]
        yield
        reads[r] = x
        if d is not None:
            newv[r] = x + d
    if not fail:
        if ts is None:                                  # lock point
            ts = m.clock
            m.clock += 1
            yield
        for (r, d) in held:
            if d is not None:
                m.val[r] = newv[r]
                yield
    for (r, d) in held:                                 # release
        m.word[r] = m.word[r] - 1 if d is None else 0
        yield
    if not fail:
        out.append(((ts,), reads))


# ---------------------------------------------------------------------------
# basic TO: timestamp at the start; a read needs a clean wts <= ts, raises
# rts to ts, loads the value and checks that wts did not move; a write needs
# ts >= rts and ts >= wts and marks the word dirty with wts = ts by a 128-bit
# CAS; writes, then wts published; an abort restores the saved wts.
# ---------------------------------------------------------------------------
DIRTY = 1 << 61


def to_txn(m, ops, out, recheck=True, write_value="before_mark"):
    """write_value: where a writer reads the record's value -- "before_mark"
    (the design: after the word, before the CAS that marks it dirty; kept if
    that CAS succeeds), "after_mark" (under the mark) or "before_word" (a
    rejected order: the value before the word it is paired with)."""
    ts = m.clock + 1
    m.clock += 1
    yield
    reads, newv, saved = {}, {}, {}
    fail = False
    for (r, d) in ops:
        if d is None:
            for tries in range(3):
                y1 = m.word[r]
                yield
                if (y1 & DIRTY) or ts < y1:
                    fail = True
                    break
                m.rts[r] = max(m.rts[r], ts)            # atomic max
                yield
                x = m.val[r]
                yield
                if not recheck or m.word[r] == y1:
                    reads[r] = x
                    break
                yield
            else:
                fail = True
        else:
            if write_value == "before_word":
                x = m.val[r]
                yield
            w_r, w_w = m.rts[r], m.word[r]              # one 128-bit load (acquire)
            yield
            if (w_w & DIRTY) or ts < w_r or ts < w_w:
                fail = True
            else:
                if write_value == "before_mark":
                    x = m.val[r]
                    yield
                if m.rts[r] == w_r and m.word[r] == w_w:    # the CAS
                    m.word[r] = DIRTY | ts
                    saved[r] = w_w
                    yield
                    if write_value == "after_mark":
                        x = m.val[r]
                        yield
                    reads[r] = x
                    newv[r] = x + d
                else:
                    fail = True
        if fail:
            break
    if fail:
        for r, w in saved.items():
            m.word[r] = w
            yield
        return
    for r in saved:
        m.val[r] = newv[r]
        yield
    for r in saved:
        m.word[r] = ts
        yield
    out.append(((ts,), reads))


def run_schedule(make_txn, scenario, initial, seed):
    """Interleave the scenario's transactions by a seeded random schedule;
    returns (committed [(order key, reads, ops)], final values)."""
    m = Mem(initial)
    outs = [[] for _ in scenario]
    gens = [make_txn(m, ops, outs[i], i) for i, ops in enumerate(scenario)]
    live = list(range(len(gens)))
    rng = random.Random(seed)
    while live:
        i = rng.choice(live)
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
    committed = []
    for i, o in enumerate(outs):
        if o:
            key, reads = o[0]
            committed.append((key, reads, scenario[i]))
    return committed, m.val


def serial_replay_ok(committed, initial, final):
    """Committed transactions in order-key order, one after another, must read
    what they read concurrently and leave the final values."""
    val = list(initial)
    for _, reads, ops in sorted(committed, key=lambda c: c[0]):
        for (r, d) in ops:
            if val[r] != reads[r]:
                return False
            if d is not None:
                val[r] += d
    return val == list(final)


# scenarios: (record, delta) per op; delta None = read
SCENARIOS = {
    "write-skew": [[(0, None), (1, 5)], [(1, None), (0, 7)]],
    "lost-update": [[(0, 1)], [(0, 2)], [(0, 4)]],
    "read-then-overwrite": [[(0, None), (1, None)], [(0, 3)], [(1, 9), (0, 1)]],
    "chains": [[(0, 1), (1, None)], [(1, 2), (2, None)], [(2, 3), (0, None)]],
    "hot-reader": [[(0, None), (2, None)], [(0, 5), (1, None)], [(2, 4), (0, None)],
                   [(0, 6)]],
}


def _count_violations(make_txn, scenario, n):
    initial = [100, 200, 300]
    bad = commits = 0
    for seed in range(n):
        committed, final = run_schedule(make_txn, scenario, initial, seed)
        commits += len(committed)
        if not serial_replay_ok(committed, initial, final):
            bad += 1
    return bad, commits


MODELS = {
    "occ": lambda m, ops, out, i: occ_txn(m, ops, out),
    "2pl": lambda m, ops, out, i: tpl_txn(m, ops, out, i),
    "2pl_wd": lambda m, ops, out, i: tpl_txn(m, ops, out, i, wait_die=True),
    "to": lambda m, ops, out, i: to_txn(m, ops, out),
    "tictoc": lambda m, ops, out, i: tictoc_txn(m, ops, out),
}


@pytest.mark.parametrize("scheme", sorted(MODELS))
@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_protocol_is_serializable(scheme, name):
    bad, commits = _count_violations(MODELS[scheme], SCENARIOS[name], 4000)
    assert bad == 0
    assert commits > 0


def test_occ_timestamp_taken_with_the_locks_is_not_serializable():
    """Negative control: a writer's timestamp can precede a reader's
    validation of the record the writer is locking."""
    make = lambda m, ops, out, i: occ_txn(m, ops, out, ticket_with_locks=True)
    bad = sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS)
    assert bad > 0


def test_tictoc_without_the_snapshot_recheck_is_not_serializable():
    """Negative control: wts read before a writer publishes, value and rts
    after, and a read covered by that rts is never checked again."""
    make = lambda m, ops, out, i: tictoc_txn(m, ops, out, recheck=False)
    bad = sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS)
    assert bad > 0


def test_2pl_ticket_before_the_lock_point_is_not_serializable():
    """Negative control: a ticket taken before the locks orders a transaction
    ahead of one whose write it then reads."""
    make = lambda m, ops, out, i: tpl_txn(m, ops, out, i, ticket_first=True)
    bad = sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS)
    assert bad > 0


def test_to_read_without_the_wts_recheck_is_not_serializable():
    """Negative control: a younger writer locks, writes and publishes between
    the read's wts check and its value load."""
    make = lambda m, ops, out, i: to_txn(m, ops, out, recheck=False)
    bad = sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS)
    assert bad > 0


def test_to_writer_value_orders():
    """The writer's value read under the mark and read before it (between
    the word and the CAS) are both serializable; read before the word, a
    writer that commits in between pairs an old value with a new word."""
    for order in ("after_mark", "before_mark"):
        make = lambda m, ops, out, i: to_txn(m, ops, out, write_value=order)
        assert sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS) == 0
    make = lambda m, ops, out, i: to_txn(m, ops, out, write_value="before_word")
    assert sum(_count_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS) > 0


def test_wait_die_lets_the_older_transaction_wait():
    """The wait-die model commits at least as often as NO_WAIT on the
    scenarios (waiting replaces some aborts) and stays serializable."""
    nw = sum(_count_violations(MODELS["2pl"], SCENARIOS[n], 2000)[1] for n in SCENARIOS)
    wd = sum(_count_violations(MODELS["2pl_wd"], SCENARIOS[n], 2000)[1] for n in SCENARIOS)
    assert wd >= nw


# ---------------------------------------------------------------------------
# Retry queues: a queue word holds (tickets taken, tickets finished).  A
# transaction takes a ticket k (the taken count before it) and is admitted
# once k - finished, as a signed distance, is below the queue width; its
# attempt then ends and counts one ticket finished.  With a width above one,
# later tickets can finish first, so the distance of a ticket that was asleep
# can be negative.
# ---------------------------------------------------------------------------
def run_queue(n, width, seed, signed=True, max_steps=20000):
    """Random interleaving of n transactions through one queue; returns
    (all served, largest number of admitted-and-unfinished tickets)."""
    rng = random.Random(seed)
    taken = finished = 0
    state = ["new"] * n
    ticket = [0] * n
    left = [0] * n
    running = peak = 0
    for _ in range(max_steps):
        live = [i for i in range(n) if state[i] != "done"]
        if not live:
            return True, peak
        i = rng.choice(live)
        if state[i] == "new":
            ticket[i] = taken
            taken += 1
            state[i] = "wait"
        if state[i] == "wait":
            d = (ticket[i] - finished) & 0xFFFFFFFF
            ahead = d - (1 << 32) if (signed and d >= 1 << 31) else d
            if ahead < width:
                state[i] = "run"
                left[i] = rng.randint(1, 4)
                running += 1
                peak = max(peak, running)
        elif state[i] == "run":
            left[i] -= 1
            if left[i] == 0:
                finished += 1
                running -= 1
                state[i] = "done"
    return False, peak


@pytest.mark.parametrize("width", [1, 2, 4])
def test_retry_queue_admits_at_most_width_and_serves_everyone(width):
    for seed in range(300):
        served, peak = run_queue(24, width, seed)
        assert served, seed
        assert peak <= width


def test_retry_queue_with_an_unsigned_distance_strands_tickets():
    """Negative control: read as unsigned, a negative distance looks huge and
    the sleeping ticket is never admitted."""
    stuck = sum(not run_queue(24, 4, seed, signed=False)[0] for seed in range(300))
    assert stuck > 0


# ---------------------------------------------------------------------------
# Multi-version TO (the TO-based MVCC of Sec. III-E, "MVCC"; a design for a
# device implementation, checked here before it is built).  Versions are
# immutable once made.  Each record has one atomically updated head word
# (wts of its newest committed version, that version's rts, the timestamp of
# a pending writer or 0).  Writes happen only at the head: a writer with
# timestamp ts needs no pending writer, wts < ts and rts <= ts, and installs
# itself as the pending writer by a CAS; at commit it creates its version and
# publishes (ts, ts, 0).  A read with timestamp ts aborts if a writer older
# than ts is pending; if the head is older than ts it raises the head's rts
# to ts by a CAS that keeps the rest of the word; otherwise it reads the
# newest version older than ts, which no later write can displace (writes go
# above the head only).  Serial order: the timestamps.
# ---------------------------------------------------------------------------
class MVMem:
    def __init__(self, values):
        self.head = [(0, 0, 0)] * len(values)           # (wts, rts, pending ts)
        self.versions = [{0: v} for v in values]        # wts -> value, immutable
        self.clock = 0


def mvto_txn(m, ops, out, raise_rts=True, check_rts=True):
    ts = m.clock + 1
    m.clock += 1
    yield
    reads, newv, pending = {}, {}, []
    fail = False
    for (r, d) in ops:
        for _ in range(3):                              # CAS retries
            w, rt, pend = m.head[r]                     # one 16-byte load
            yield
            if d is None:
                if pend and pend < ts:
                    fail = True
                    break
                if w < ts:
                    if raise_rts:
                        if m.head[r] != (w, rt, pend):  # the CAS
                            yield
                            continue
                        m.head[r] = (w, max(rt, ts), pend)
                        yield
                    reads[r] = m.versions[r][w]
                else:
                    older = max(k for k in m.versions[r] if k < ts)
                    reads[r] = m.versions[r][older]
                yield
                break
            if pend or w >= ts or (check_rts and rt > ts):
                fail = True
                break
            if m.head[r] != (w, rt, pend):              # the CAS
                yield
                continue
            m.head[r] = (w, rt, ts)
            pending.append(r)
            yield
            reads[r] = m.versions[r][w]
            newv[r] = reads[r] + d
            yield
            break
        else:
            fail = True
        if fail:
            break
    if fail:
        for r in pending:                               # withdraw, keeping rts raises
            w, rt, _ = m.head[r]
            m.head[r] = (w, rt, 0)
            yield
        return
    for r in pending:
        m.versions[r][ts] = newv[r]                     # the new version, then publish
        yield
        m.head[r] = (ts, ts, 0)
        yield
    out.append(((ts,), reads))


def run_mv_schedule(make_txn, scenario, initial, seed):
    m = MVMem(initial)
    outs = [[] for _ in scenario]
    gens = [make_txn(m, ops, outs[i]) for i, ops in enumerate(scenario)]
    live = list(range(len(gens)))
    rng = random.Random(seed)
    while live:
        i = rng.choice(live)
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
    committed = [(o[0][0], o[0][1], scenario[i]) for i, o in enumerate(outs) if o]
    final = [m.versions[r][m.head[r][0]] for r in range(len(initial))]
    return committed, final


def _mv_violations(make_txn, scenario, n):
    initial = [100, 200, 300]
    bad = commits = 0
    for seed in range(n):
        committed, final = run_mv_schedule(make_txn, scenario, initial, seed)
        commits += len(committed)
        if not serial_replay_ok(committed, initial, final):
            bad += 1
    return bad, commits


@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_mvto_design_is_serializable(name):
    bad, commits = _mv_violations(mvto_txn, SCENARIOS[name], 4000)
    assert bad == 0
    assert commits > 0


def test_mvto_old_readers_do_not_abort_on_newer_versions():
    """The point of the versions: a reader older than the head commits where
    single-version TO aborts it."""
    sc = SCENARIOS["read-then-overwrite"]
    mv = _mv_violations(mvto_txn, sc, 3000)[1]
    to = _count_violations(MODELS["to"], sc, 3000)[1]
    assert mv > to


@pytest.mark.parametrize("variant", [dict(raise_rts=False), dict(check_rts=False)])
def test_mvto_without_the_read_timestamp_is_not_serializable(variant):
    """Negative controls: a read that does not raise the head's rts, or a
    writer that ignores it, lets a writer older than a reader slip under it."""
    make = lambda m, ops, out: mvto_txn(m, ops, out, **variant)
    bad = sum(_mv_violations(make, SCENARIOS[n], 4000)[0] for n in SCENARIOS)
    assert bad > 0


# ---------------------------------------------------------------------------
# OCC with early write locks on hot records (a design for shortening the
# hot-record chain, checked before it is built): a write to a record marked
# hot takes its lock before reading it, waiting a bounded number of steps for
# the holder and aborting after that; every other access follows OCC above.
# The timestamp is still taken after all write locks and before validation.
# ---------------------------------------------------------------------------
def occ_early_txn(m, ops, out, hot=frozenset({0}), wait_steps=6):
    obs, reads, newv = {}, {}, {}
    held = []

    def release():
        for h in held:
            m.word[h] = obs[h]

    for (r, d) in ops:
        if d is not None and r in hot:
            for _ in range(wait_steps + 1):             # lock first, bounded wait
                v = m.word[r]
                if not (v & LOCK):
                    m.word[r] = v | LOCK                # the CAS
                    obs[r] = v
                    held.append(r)
                    yield
                    break
                yield
            else:
                release()
                return
            x = m.val[r]                                # read under the lock
            yield
            reads[r], newv[r] = x, x + d
            continue
        v1 = m.word[r]
        yield
        if v1 & LOCK:
            release()
            return
        x = m.val[r]
        yield
        obs[r], reads[r] = v1, x
        if d is not None:
            newv[r] = x + d
    for (r, d) in ops:                                  # the other write locks
        if d is None or r in held:
            continue
        if m.word[r] != obs[r]:
            release()
            return
        m.word[r] = obs[r] | LOCK
        held.append(r)
        yield
    ts = m.clock
    m.clock += 1
    yield
    for (r, d) in ops:
        if d is None:
            ok = m.word[r] == obs[r]
            yield
            if not ok:
                release()
                return
    for r in held:
        m.val[r] = newv[r]
        yield
    for r in held:
        m.word[r] = ts + 1
        yield
    out.append(((ts,), reads))


@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_occ_with_early_hot_locks_is_serializable(name):
    make = lambda m, ops, out, i: occ_early_txn(m, ops, out)
    bad, commits = _count_violations(make, SCENARIOS[name], 4000)
    assert bad == 0
    assert commits > 0


def test_occ_early_hot_locks_commit_more_on_the_hot_record():
    """Writers of the hot record wait for it instead of failing validation:
    more commits than plain OCC where they collide."""
    make = lambda m, ops, out, i: occ_early_txn(m, ops, out)
    for name in ("lost-update", "hot-reader"):
        early = _count_violations(make, SCENARIOS[name], 3000)[1]
        plain = _count_violations(MODELS["occ"], SCENARIOS[name], 3000)[1]
        assert early > plain, name


# ---------------------------------------------------------------------------
# The same multi-version TO at the level of the planned device structures.
# Control words are per record (conflicts at record granularity), values per
# (record, field) slot.  A record's 16-byte head word is (wts, rts, pending
# writer, chain), timestamps batch-relative.  Committed writes append
# immutable entries (wts, field, value, next) to a batch-wide version store
# (an atomic counter hands out indices), and chain is the newest entry's
# index + 1 (0: none, the table slot is the record's only version).
#
# A read of field f at ts:
#   - if the head is older than ts, it raises rts by a CAS;
#   - it then takes the newest entry older than ts that wrote f, walking the
#     chain from the head, or else the table slot, which nothing writes
#     during the batch.
#
# At the batch's end a flatten pass writes each slot's newest entry into the
# table and zeroes the heads.
# ---------------------------------------------------------------------------
class DevMV:
    def __init__(self, table):                          # table[record][field]
        self.table = [list(r) for r in table]
        self.head = [(0, 0, 0, 0)] * len(table)         # (wts, rts, pend, chain)
        self.store = []                                 # (wts, field, value, next)
        self.clock = 0


def _dev_value(m, r, f, chain, ts):
    e = chain
    while e:
        wts, field, value, nxt = m.store[e - 1]
        if wts < ts and field == f:
            return value
        e = nxt
    return m.table[r][f]


def dev_mvto_txn(m, ops, out, raise_by_max=False):
    """ops: (record, field, delta or None).  raise_by_max: a reader raises
    rts by an atomic max on its own 32-bit field (which never fails) and then
    reads the head again, retrying if wts, the pending mark or the chain moved
    -- instead of one CAS over the whole head."""
    m.clock += 1
    ts = m.clock
    yield
    reads, pending = {}, {}
    fail = False
    for (r, f, d) in ops:
        for _ in range(3):
            h = m.head[r]                               # one 16-byte load
            w, rt, pend, chain = h
            yield
            if d is None:
                if pend and pend < ts:
                    fail = True
                    break
                if w < ts and raise_by_max:
                    cw, crt, cp, cc = m.head[r]         # atomic max on the rts field
                    m.head[r] = (cw, max(crt, ts), cp, cc)
                    yield
                    w2, _, p2, c2 = m.head[r]           # the head again
                    yield
                    if (w2, p2, c2) != (w, pend, chain):
                        continue
                elif w < ts:
                    if m.head[r] != h:                  # CAS raising rts
                        yield
                        continue
                    m.head[r] = (w, max(rt, ts), pend, chain)
                    yield
                reads[(r, f)] = _dev_value(m, r, f, chain, ts)
                yield
                break
            if pend or w >= ts or rt > ts:
                fail = True
                break
            if m.head[r] != h:                          # CAS installing the pending writer
                yield
                continue
            m.head[r] = (w, rt, ts, chain)
            old = _dev_value(m, r, f, chain, ts)
            yield
            reads[(r, f)] = old
            pending[r] = (f, old + d)
            break
        else:
            fail = True
        if fail:
            break
    if fail:
        for r in pending:                               # withdraw by CAS loop
            w, rt, _, chain = m.head[r]
            m.head[r] = (w, rt, 0, chain)
            yield
        return
    for r, (f, v) in pending.items():
        m.store.append(None)                            # index from the counter
        idx = len(m.store)
        yield
        m.store[idx - 1] = (ts, f, v, m.head[r][3])     # the entry, then publish
        yield
        m.head[r] = (ts, ts, 0, idx)                    # CAS loop: only rts can move
        yield
    out.append(((ts,), reads))


def dev_flatten(m):
    for r, (_, _, _, chain) in enumerate(m.head):
        seen = set()
        e = chain
        while e:
            wts, f, v, nxt = m.store[e - 1]
            if f not in seen:
                m.table[r][f] = v
                seen.add(f)
            e = nxt
        m.head[r] = (0, 0, 0, 0)
    m.store.clear()


DEV_SCENARIOS = {
    "fields of one record": [[(0, 0, None), (1, 1, 5)], [(0, 1, 3)], [(0, 0, 2), (1, 0, None)]],
    "write skew": [[(0, 0, None), (1, 0, 4)], [(1, 0, None), (0, 0, 6)]],
    "hot record": [[(0, 0, 1)], [(0, 1, 2)], [(0, 0, None), (1, 1, 7)], [(0, 0, 3), (1, 1, None)]],
    "old reader behind other fields": [[(0, 0, 1)], [(0, 1, 2)], [(0, 0, None)], [(0, 0, 3)],
                                       [(0, 1, 4)], [(0, 1, None)]],
}


def _dev_replay(committed, initial, final):
    val = [list(r) for r in initial]
    for _, reads, ops in sorted(committed, key=lambda c: c[0]):
        for (r, f, d) in ops:
            if val[r][f] != reads[(r, f)]:
                return False
            if d is not None:
                val[r][f] += d
    return val == final


def _dev_runs(scenario, n, flatten=None, raise_by_max=False):
    """(violations, commits) over n seeded interleavings, flattened at the end."""
    initial = [[100, 200], [300, 400]]
    bad = commits = 0
    for seed in range(n):
        m = DevMV(initial)
        outs = [[] for _ in scenario]
        gens = [dev_mvto_txn(m, ops, outs[i], raise_by_max) for i, ops in enumerate(scenario)]
        live = list(range(len(gens)))
        rng = random.Random(seed)
        while live:
            i = rng.choice(live)
            try:
                next(gens[i])
            except StopIteration:
                live.remove(i)
        (flatten or dev_flatten)(m)
        assert m.head == [(0, 0, 0, 0)] * len(initial) and not m.store
        committed = [(o[0][0], o[0][1], scenario[i]) for i, o in enumerate(outs) if o]
        commits += len(committed)
        bad += not _dev_replay(committed, initial, m.table)
    return bad, commits


@pytest.mark.parametrize("raise_by_max", [False, True])
@pytest.mark.parametrize("name", sorted(DEV_SCENARIOS))
def test_device_mvto_layout_is_serializable(name, raise_by_max):
    bad, commits = _dev_runs(DEV_SCENARIOS[name], 3000, raise_by_max=raise_by_max)
    assert bad == 0
    assert commits > 0


def test_device_mvto_max_raise_needs_the_second_look(monkeypatch):
    """Negative control: raising rts by max without reading the head again
    lets a writer that installed itself in between slip under the reader."""
    def blind(m, ops, out):
        m.clock += 1
        ts = m.clock
        yield
        reads, pending = {}, {}
        for (r, f, d) in ops:
            w, rt, pend, chain = m.head[r]
            yield
            if d is None:
                if pend and pend < ts:
                    break
                if w < ts:
                    cw, crt, cp, cc = m.head[r]
                    m.head[r] = (cw, max(crt, ts), cp, cc)
                    yield
                reads[(r, f)] = _dev_value(m, r, f, chain, ts)
                yield
                continue
            if pend or w >= ts or rt > ts or m.head[r] != (w, rt, pend, chain):
                break
            m.head[r] = (w, rt, ts, chain)
            reads[(r, f)] = old = _dev_value(m, r, f, chain, ts)
            pending[r] = (f, old + d)
            yield
        else:
            for r, (f, v) in pending.items():
                m.store.append(None)
                idx = len(m.store)
                yield
                m.store[idx - 1] = (ts, f, v, m.head[r][3])
                yield
                m.head[r] = (ts, ts, 0, idx)
                yield
            out.append(((ts,), reads))
            return
        for r in pending:
            w, rt, _, chain = m.head[r]
            m.head[r] = (w, rt, 0, chain)
            yield
    monkeypatch.setattr(sys.modules[__name__], "dev_mvto_txn", lambda m, o, out, rbm=False: blind(m, o, out))
    bad = sum(_dev_runs(DEV_SCENARIOS[n], 3000)[0] for n in DEV_SCENARIOS)
    assert bad > 0


def test_device_mvto_flatten_must_take_the_newest_entry(monkeypatch):
    """Negative control: a flatten that lets the oldest entry of a slot win."""
    def oldest_wins(m):
        for r, (_, _, _, chain) in enumerate(m.head):
            e = chain
            while e:
                _, f, v, nxt = m.store[e - 1]
                m.table[r][f] = v
                e = nxt
            m.head[r] = (0, 0, 0, 0)
        m.store.clear()
    assert _dev_runs(DEV_SCENARIOS["old reader behind other fields"], 3000, oldest_wins)[0] > 0


def test_device_mvto_walk_must_match_the_field(monkeypatch):
    """Negative control: a walk that stops at the first entry older than the
    reader whatever field it wrote."""
    def first_older(m, r, f, chain, ts):
        e = chain
        while e:
            wts, field, value, nxt = m.store[e - 1]
            if wts < ts:
                return value if field == f else m.table[r][f]
            e = nxt
        return m.table[r][f]
    monkeypatch.setattr(sys.modules[__name__], "_dev_value", first_older)
    assert _dev_runs(DEV_SCENARIOS["old reader behind other fields"], 3000)[0] > 0


# ---------------------------------------------------------------------------
# MVCC as the kernel builds it: concurrency control per record in a head word
# (wts, rts, pending writer), versions per (record, field) slot.  A slot's
# version pointer names its newest entry in the batch's version store; each
# entry (wts, next, record, field, value) links to the slot's previous one.
# A write at ts installs itself as the record's pending writer by a CAS
# (needs no pending writer, wts < ts, rts <= ts) and reads its slot's newest
# version in one step (the pointer's entry, or the table slot).  A read at ts
# aborts on an older pending writer, raises rts by a CAS when the record's
# newest version is older than ts, then walks its slot's entries from the
# newest to the first older than ts.  Commit: entries, then pointers, then
# heads (ts, ts, 0).  At the batch's end every slot's newest entry goes into
# the table and pointers and heads are cleared.
# ---------------------------------------------------------------------------
class SlotMV:
    def __init__(self, table):                          # table[record][field]
        self.table = [list(r) for r in table]
        self.head = [(0, 0, 0)] * len(table)            # (wts, rts, pend)
        self.slot = {}                                  # (r, f) -> entry index + 1
        self.store = []                                 # (wts, next, r, f, value)
        self.clock = 0


def _slot_value(m, r, f, ts, e=None):
    """The newest version of slot (r, f) older than ts, walking from pointer e
    (read now when not given)."""
    if e is None:
        e = m.slot.get((r, f), 0)
    while e:
        wts, nxt, _, _, value = m.store[e - 1]
        if wts < ts:
            return value
        e = nxt
    return m.table[r][f]


def slot_mvto_txn(m, ops, out, pointers_before_heads=True, writer_reads_table=False,
                  reads_before_mark=True, versions_before_head=False):
    """reads_before_mark (the design): a writer reads its slot's newest version
    after the head and before the CAS that installs it as pending (kept if
    that CAS succeeds), and a reader takes its slot's pointer before the CAS
    that raises rts.  versions_before_head: the rejected order, the version
    read before the head it is checked against."""
    m.clock += 1
    ts = m.clock
    yield
    reads, pending = {}, {}
    fail = False
    def newest(r, f):                                   # pointer, then its entry or the table
        e = m.slot.get((r, f), 0)
        return e, (m.table[r][f] if (writer_reads_table or not e) else m.store[e - 1][4])

    for (r, f, d) in ops:
        for _ in range(3):
            if versions_before_head:
                pe = m.slot.get((r, f), 0)
                e, old = newest(r, f)
                yield
            h = m.head[r]                               # one 16-byte load
            w, rt, pend = h
            yield
            if d is None:
                if pend and pend < ts:
                    fail = True
                    break
                if reads_before_mark and not versions_before_head:
                    pe = m.slot.get((r, f), 0)          # the pointer beside the rts CAS
                    yield
                if w < ts and rt < ts:
                    if m.head[r] != h:                  # CAS raising rts
                        yield
                        continue
                    m.head[r] = (w, ts, pend)
                    yield
                if reads_before_mark or versions_before_head:
                    reads[(r, f)] = _slot_value(m, r, f, ts, pe)
                else:
                    reads[(r, f)] = _slot_value(m, r, f, ts)
                yield
                break
            if pend or w >= ts or rt > ts:
                fail = True
                break
            if reads_before_mark and not versions_before_head:
                e, old = newest(r, f)
                yield
            if m.head[r] != h:                          # CAS installing the pending writer
                yield
                continue
            m.head[r] = (w, rt, ts)
            yield
            if not reads_before_mark and not versions_before_head:
                e, old = newest(r, f)
                yield
            reads[(r, f)] = old
            pending[r] = (f, old + d, e)
            break
        else:
            fail = True
        if fail:
            break
    if fail:
        for r in pending:                               # withdraw by CAS loop
            w, rt, _ = m.head[r]
            m.head[r] = (w, rt, 0)
            yield
        return
    idx = {}
    for r, (f, v, prev) in pending.items():
        m.store.append((ts, prev, r, f, v))             # the entry
        idx[r] = len(m.store)
        yield

    def pointers():
        for r, (f, _, _) in pending.items():
            m.slot[(r, f)] = idx[r]
            yield

    def heads():
        for r in pending:                               # CAS loop: only rts can move
            _, rt, _ = m.head[r]
            m.head[r] = (ts, max(rt, ts), 0)
            yield

    steps = (pointers, heads) if pointers_before_heads else (heads, pointers)
    for part in steps:
        yield from part()
    out.append(((ts,), reads))


def slot_flatten(m):
    for i, (_, _, r, f, v) in enumerate(m.store):
        if m.slot.get((r, f)) == i + 1:
            m.table[r][f] = v
            del m.slot[(r, f)]
    m.head = [(0, 0, 0)] * len(m.head)
    m.store.clear()


def _slot_runs(scenario, n, **kw):
    initial = [[100, 200], [300, 400]]
    bad = commits = 0
    for seed in range(n):
        m = SlotMV(initial)
        outs = [[] for _ in scenario]
        gens = [slot_mvto_txn(m, ops, outs[i], **kw) for i, ops in enumerate(scenario)]
        live = list(range(len(gens)))
        rng = random.Random(seed)
        while live:
            i = rng.choice(live)
            try:
                next(gens[i])
            except StopIteration:
                live.remove(i)
        slot_flatten(m)
        assert not m.slot and not m.store
        committed = [(o[0][0], o[0][1], scenario[i]) for i, o in enumerate(outs) if o]
        commits += len(committed)
        bad += not _dev_replay(committed, initial, m.table)
    return bad, commits


@pytest.mark.parametrize("name", sorted(DEV_SCENARIOS))
def test_slot_mvcc_layout_is_serializable(name):
    bad, commits = _slot_runs(DEV_SCENARIOS[name], 3000)
    assert bad == 0
    assert commits > 0


def test_slot_mvcc_reads_under_the_mark_are_serializable_too():
    """The earlier order (a writer reads its slot's newest version after the
    pending mark, a reader its pointer after the rts raise) replays as well."""
    for n in DEV_SCENARIOS:
        bad, commits = _slot_runs(DEV_SCENARIOS[n], 2000, reads_before_mark=False)
        assert bad == 0 and commits > 0


@pytest.mark.parametrize("variant", [dict(pointers_before_heads=False),
                                     dict(writer_reads_table=True),
                                     dict(versions_before_head=True)],
                         ids=["heads before pointers", "writer reads the table slot",
                              "versions read before the head"])
def test_slot_mvcc_negative_controls(variant):
    """A head published before its slots' pointers lets a newer reader take a
    superseded version; a writer that reads the table slot instead of the
    slot's newest version loses updates; a version read before the head it is
    checked against can be superseded by a commit in between.  Each must
    produce violations."""
    bad = sum(_slot_runs(DEV_SCENARIOS[n], 3000, **variant)[0] for n in DEV_SCENARIOS)
    assert bad > 0


# ---------------------------------------------------------------------------
# Whole batches with retries, in parallel rounds: every live transaction
# takes one memory step per round (the GPU runs them side by side); an
# aborted one restarts after a randomized backoff (rounds, doubling with its
# aborts).  With early locks, a transaction that aborted on a record it
# writes locks that record in its next attempts (occ_retry_txn below mirrors
# the early-lock kernel: the record is locked after the read phase, with a
# bounded wait).  The histories must replay, and the round count compares
# the two policies on a batch with one hot record.
# ---------------------------------------------------------------------------
def occ_retry_txn(m, ops, out, info, early=None, wait_steps=64):
    obs, reads, newv, held = {}, {}, {}, []

    def release():
        for h in held:
            m.word[h] = obs[h]

    for (r, d) in ops:
        if r == early and d is not None:
            continue                                    # read under its lock below
        v1 = m.word[r]
        yield
        if v1 & LOCK:
            info["crec"] = r
            return
        x = m.val[r]
        yield
        obs[r], reads[r] = v1, x
        if d is not None:
            newv[r] = x + d
    de = next((d for r, d in ops if r == early and d is not None), None)
    if de is not None:
        for _ in range(wait_steps + 1):
            v = m.word[early]
            if not (v & LOCK):
                m.word[early] = v | LOCK                # the CAS
                obs[early] = v
                held.append(early)
                yield
                break
            yield
        else:
            info["crec"] = early
            return
        x = m.val[early]
        yield
        reads[early], newv[early] = x, x + de
    for (r, d) in ops:
        if d is None or r in held:
            continue
        if m.word[r] != obs[r]:
            info["crec"] = r
            release()
            return
        m.word[r] = obs[r] | LOCK
        held.append(r)
        yield
    ts = m.clock
    m.clock += 1
    yield
    for (r, d) in ops:
        if d is None:
            ok = m.word[r] == obs[r]
            yield
            if not ok:
                info["crec"] = r
                release()
                return
    for r in held:
        m.val[r] = newv[r]
        yield
    for r in held:
        m.word[r] = ts + 1
        yield
    out.append(((ts,), reads))


def run_batch_rounds(txns, nrec, seed, early_after=0, max_rounds=100000):
    """(rounds to commit everything, aborts, history replays, committed)."""
    rng = random.Random(seed)
    initial = [100 + i for i in range(nrec)]
    m = Mem(initial)
    n = len(txns)
    outs = [[] for _ in range(n)]
    state, info = [None] * n, [dict() for _ in range(n)]
    aborts, early = [0] * n, [None] * n

    def start(i):
        info[i] = {}
        state[i] = occ_retry_txn(m, txns[i], outs[i], info[i], early[i])

    for i in range(n):
        start(i)
    done = rounds = 0
    while done < n and rounds < max_rounds:
        rounds += 1
        order = list(range(n))
        rng.shuffle(order)
        for i in order:
            s = state[i]
            if s is None:
                continue
            if isinstance(s, int):                      # backing off until round s
                if rounds >= s:
                    start(i)
                continue
            try:
                next(s)
            except StopIteration:
                if outs[i]:
                    state[i] = None
                    done += 1
                    continue
                aborts[i] += 1
                c = info[i].get("crec")
                if (early_after and c is not None and aborts[i] >= early_after
                        and any(r == c and d is not None for r, d in txns[i])):
                    early[i] = c
                state[i] = rounds + 1 + rng.randint(0, min(1 << min(aborts[i], 10), 64))
    committed = [(outs[i][0][0], outs[i][0][1], txns[i]) for i in range(n) if outs[i]]
    return rounds, sum(aborts), serial_replay_ok(committed, initial, m.val), done


def hot_batch(seed, n=96, nrec=64, ops=4, hot_share=0.5, read_ratio=0.5):
    """Transactions of `ops` distinct records; record 0 is in `hot_share` of them."""
    rng = random.Random(seed)
    txns = []
    for _ in range(n):
        keys = {0} if rng.random() < hot_share else set()
        while len(keys) < ops:
            keys.add(rng.randrange(1, nrec))
        txns.append([(k, None if rng.random() < read_ratio else rng.randint(1, 9))
                     for k in sorted(keys)])
    return txns


@pytest.mark.parametrize("early_after", [0, 1, 3])
def test_batches_with_retries_replay(early_after):
    for seed in range(6):
        rounds, aborts, ok, done = run_batch_rounds(hot_batch(seed), 64, seed, early_after)
        assert ok and done == 96, (seed, rounds, aborts)


def test_early_locks_take_fewer_rounds_on_a_hot_batch():
    """In the round model, early locks shorten the hot record's chain more
    than they delay its readers (read ratios 0.5 and 0: writers dominate)."""
    for rr in (0.5, 0.0):
        plain = sum(run_batch_rounds(hot_batch(s, read_ratio=rr), 64, s, 0)[0] for s in range(6))
        early = sum(run_batch_rounds(hot_batch(s, read_ratio=rr), 64, s, 1)[0] for s in range(6))
        assert early < plain, (rr, early, plain)


# ---------------------------------------------------------------------------
# OCC group commit (key-value batches): a unit of member transactions runs as
# one attempt -- every member's reads (version, then value), one lock CAS per
# distinct written record from the version its lowest op saw, consecutive
# timestamps for the members still in, per-member validation of the reads of
# records the unit does not hold, then each held record evaluated in member
# order over the committing members (a member's read returns the value after
# the earlier members' writes), written once and published once with the
# last writer's timestamp + 1.  Units and single OCC transactions interleave
# on the same records; every committed member, replayed in timestamp order,
# must read what it read.  The negative control drops the composition: each
# member reads and adds to the value its own read saw.
# ---------------------------------------------------------------------------
def occ_unit_txn(m, members, outs, compose=True):
    ops_all = [(mi, r, d) for mi, ops in enumerate(members) for (r, d) in ops]
    obs, val = {}, {}
    dead = set()
    for k, (mi, r, d) in enumerate(ops_all):            # read phase
        v1 = m.word[r]
        yield
        if v1 & LOCK:
            dead.add(mi)
            continue
        val[k] = m.val[r]
        obs[k] = v1
        yield
    rep = {}
    for k, (mi, r, d) in enumerate(ops_all):            # lowest op per record
        rep.setdefault(r, k)
    written = sorted({r for (_, r, d) in ops_all if d is not None})
    held = {}
    for r in written:                                    # one lock CAS per record
        k = rep[r]
        if k in obs and m.word[r] == obs[k]:
            m.word[r] = obs[k] | LOCK
            held[r] = obs[k]
        yield
    for (mi, r, d) in ops_all:
        if d is not None and r not in held:
            dead.add(mi)
    alive = [mi for mi in range(len(members)) if mi not in dead]
    ts_of = {}
    if alive:
        base = m.clock                                   # one atomic for all of them
        m.clock += len(alive)
        ts_of = {mi: base + i for i, mi in enumerate(alive)}
        yield
        for k, (mi, r, d) in enumerate(ops_all):         # validate reads not held
            if mi in ts_of and r not in held:
                ok = m.word[r] == obs[k]
                yield
                if not ok:
                    dead.add(mi)
    won = [mi for mi in alive if mi not in dead]
    reads = {mi: {} for mi in won}
    for k, (mi, r, d) in enumerate(ops_all):
        if mi in reads and r not in held:
            reads[mi][r] = val[k]
    for r, v0 in held.items():                           # each held record, member order
        cur, last = val[rep[r]], None
        for mi in won:
            for k, (mj, rr, d) in enumerate(ops_all):
                if mj != mi or rr != r:
                    continue
                seen = cur if compose else val[k]
                reads[mi][r] = seen
                if d is not None:
                    cur = seen + d
                    last = ts_of[mi]
        if last is not None:
            m.val[r] = cur
            yield
            m.word[r] = last + 1
        else:
            m.word[r] = v0
        yield
    for mi in won:
        outs[mi].append(((ts_of[mi],), reads[mi]))


def run_actors(actors, initial, seed, compose=True):
    """Interleave units and single OCC transactions; returns (committed
    [(order key, reads, ops)], final values)."""
    m = Mem(initial)
    gens, members = [], []
    for kind, body in actors:
        if kind == "unit":
            outs = [[] for _ in body]
            gens.append(occ_unit_txn(m, body, outs, compose))
            members += list(zip(body, outs))
        else:
            out = []
            gens.append(occ_txn(m, body, out))
            members.append((body, out))
    live = list(range(len(gens)))
    rng = random.Random(seed)
    while live:
        i = rng.choice(live)
        try:
            next(gens[i])
        except StopIteration:
            live.remove(i)
    committed = [(o[0][0], o[0][1], ops) for ops, o in members if o]
    return committed, m.val


UNIT_SCENARIOS = {
    "unit-vs-singles": [("unit", [[(0, 1), (1, None)], [(0, 2)]]),
                        ("txn", [(0, 4), (1, 3)]), ("txn", [(1, None), (0, None)])],
    "two-units": [("unit", [[(0, 1)], [(0, 2), (2, None)]]),
                  ("unit", [[(0, 3), (1, None)], [(0, 4)]]), ("txn", [(2, 5)])],
    "readers-inside": [("unit", [[(0, None), (1, 1)], [(0, 2)], [(1, None)]]),
                       ("txn", [(0, 7)]), ("txn", [(1, None), (0, None)])],
    "shared-others": [("unit", [[(0, 1), (2, 1)], [(0, 2), (2, None)], [(0, 3), (1, 5)]]),
                      ("txn", [(2, 4), (1, None)])],
}


def _unit_violations(scenario, n, compose=True):
    initial = [100, 200, 300]
    bad = commits = 0
    for seed in range(n):
        committed, final = run_actors(scenario, initial, seed, compose)
        commits += len(committed)
        bad += not serial_replay_ok(committed, initial, final)
    return bad, commits


@pytest.mark.parametrize("name", sorted(UNIT_SCENARIOS))
def test_occ_group_commit_unit_is_serializable(name):
    bad, commits = _unit_violations(UNIT_SCENARIOS[name], 3000)
    assert bad == 0
    assert commits > 0


def test_occ_group_commit_commits_several_members_per_tenure():
    """Run alone, a unit commits every member in one tenure of the shared
    record: the record's version moves once, by the last member's timestamp."""
    m = Mem([100, 200, 300])
    members = [[(0, 1)], [(0, 2), (1, None)], [(0, 4)]]
    outs = [[] for _ in members]
    for _ in occ_unit_txn(m, members, outs):
        pass
    assert all(outs)
    assert m.val[0] == 107 and m.word[0] == 3            # timestamps 0, 1, 2
    assert [o[0][1][0] for o in outs] == [100, 101, 103]


def test_occ_group_commit_without_composition_is_not_serializable():
    """Negative control: members that each read and add to their own read of
    the shared record lose one another's writes."""
    bad = sum(_unit_violations(UNIT_SCENARIOS[n], 3000, compose=False)[0] for n in UNIT_SCENARIOS)
    assert bad > 0
