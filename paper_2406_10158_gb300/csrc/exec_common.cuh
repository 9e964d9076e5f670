// exec_common.cuh -- the execute kernel shared by every schema.
//
// A persistent kernel: a warp is split into lane groups of G lanes; each
// group owns one transaction at a time, taken from a global counter in
// transaction-id order (one atomic per warp and chunk of ids).  Op j of a transaction is
// handled by lane j mod G, so a group issues up to G independent record
// accesses at once, and group-wide decisions (abort, commit) are ballots over
// the group.  Per-op state -- descriptor, observed control word, value read,
// value to write -- is staged in shared memory, so an aborted attempt never
// touches the output arrays.
//
// The groups of a warp advance in rounds.  In a round every group that holds
// a transaction and is neither backing off nor waiting in a retry queue makes
// one attempt.  An aborted transaction backs off until a global-timer
// deadline drawn at random from a window that doubles with its abort count;
// after queue_after aborts it then also waits its turn in a FIFO queue of the
// record it conflicted on.  A warp with no group attempting sleeps until its
// earliest deadline.  Locks, dirty bits and write locks are only ever held
// inside an attempt, so a sleeping warp never holds any.  A transaction
// restarts until it commits (Sec. IV-A, "Experimental Procedure"), within an
// attempt budget and a kernel deadline.  Ordering between transactions rests
// on acquire/release operations: lock acquisitions acquire, unlocks and
// publishes release, OCC's commit timestamp is acquire-release.
//
// Schemes (Sec. II and Sec. III-E; control-word layouts in engine.cuh):
//  * NO_WAIT 2PL  -- shared/exclusive lock per record taken before the access,
//    abort as soon as a lock is unavailable, all locks released at commit or
//    abort (Sec. II-A, Sec. III-E.1).  Writes are buffered and applied while
//    the exclusive locks are held.  Commit order: a counter taken while every
//    lock is held (the lock point).
//  * TO           -- per-record RTS/WTS; a read needs ts > WTS, a write needs
//    ts > RTS and ts > WTS, otherwise abort and restart with a new timestamp;
//    a dirty bit locks uncommitted writes (Sec. II-B, Sec. III-E.2).  Commit
//    order: the timestamp.
//  * OCC          -- read phase into a private workspace with version checks,
//    lock the write set without waiting (abort if locked), take a commit
//    timestamp, validate the read set, write and release with the new version
//    (Sec. II-B, Sec. III-E.2 Silo: lock bit + 63-bit timestamp, no epochs,
//    no-wait locking).  Commit order: the timestamp.
//  * 2PL wait-die -- as NO_WAIT 2PL, but a transaction waits (bounded) for
//    an exclusive lock held by a younger one, and dies otherwise (Sec. II-A,
//    tpl_wd).  Commit order: the lock-point counter.
//  * TicToc       -- OCC whose commit timestamp is computed from per-record
//    write and read timestamps instead of a shared clock; a read stays valid
//    by extending its record's read timestamp (Table I lists TicToc among the
//    CPU-oriented schemes).  Commit order: (timestamp, sequence number).
//  * MVCC         -- multi-version TO: writes make versions in a batch store,
//    a read takes the newest version older than its timestamp (Sec. II,
//    Sec. III-E "MVCC").  Commit order: the timestamp.
//  * DET          -- every op waits until the lower-id accesses to its record
//    that conflict with it are done, then runs; nothing aborts and the outcome
//    is the serial execution in transaction-id order (Sec. II-C GPUTx;
//    Sec. III-E.3 access tables).  Commit order: transaction id.
//
// A workload policy `Work` supplies the record layout:
//   valid_txn(a, tx), valid_op(a, d), rec(a, d) (control word, or NO_CC),
//   writes(d), load(a, d), compute(a, d, old, operand), store(a, d, new),
//   commit_step(a, L, S, t, first, nops) (work after commit, e.g. inserts).
#pragma once

#include "engine.cuh"

namespace gcc {

constexpr uint32_t NO_CC = 0xffffffffu;     // an op on data that never changes

__device__ __forceinline__ uint32_t op_key(uint64_t d) { return (uint32_t)d; }
__device__ __forceinline__ uint32_t op_field(uint64_t d) { return (uint32_t)(d >> 32) & 0xffu; }
__device__ __forceinline__ uint32_t op_kind(uint64_t d) { return (uint32_t)(d >> 40) & 0xffu; }

struct Stage {
    uint64_t* desc;
    uint64_t* obs;
    ulonglong2* oldv;
    ulonglong2* newv;
    uint64_t* aux;           // TicToc: the record's rts as read, then as locked
};

struct Lane {
    uint32_t lane, lig, G, gbase;
    unsigned gmask;
    mutable uint32_t n_atom = 0;   // global atomic operations this lane issued
};

// SKIPPED: DET only, an invalid transaction's accesses were stepped over
enum { ABORT = 0, COMMIT = 1, GIVE_UP = 2, SKIPPED = 3 };

__device__ __forceinline__ bool collapse_loser(const ExecArgs& a, uint32_t rec) {
    if (a.collapse != 1) return false;
    const unsigned am = __activemask();
    const unsigned peers = __match_any_sync(am, rec);
    return (peers & lanemask_lt()) != 0;
}

__device__ __forceinline__ bool injected_abort(const ExecArgs& a, uint32_t t, uint32_t attempt) {
    if (a.inject_ppm == 0) return false;
    const uint64_t h = mix64(a.seed ^ (0x9E3779B97F4A7C15ull * (t + 1)) ^ ((uint64_t)attempt << 40));
    return (uint32_t)(h % 1000000ull) < a.inject_ppm;
}

// The record an aborted attempt conflicted on (the lowest failing lane's), or
// NO_CC when it aborted for another reason.  Called by every lane of the group.
__device__ __forceinline__ uint32_t group_conflict(const Lane& L, uint32_t frec) {
    const unsigned b = __ballot_sync(L.gmask, frec != NO_CC);
    if (!b) return NO_CC;
    return __shfl_sync(L.gmask, frec, __ffs(b) - 1);
}

__device__ __forceinline__ unsigned long long group_ticket(const Lane& L, unsigned long long* ctr) {
    unsigned long long v = 0;
    if (L.lig == 0) v = agg_ticket(ctr, 1, &L.n_atom);
    return __shfl_sync(L.gmask, v, L.gbase);
}
__device__ __forceinline__ unsigned long long group_ticket_acq_rel(const Lane& L,
                                                                   unsigned long long* ctr) {
    unsigned long long v = 0;
    if (L.lig == 0) v = agg_ticket_acq_rel(ctr, &L.n_atom);
    return __shfl_sync(L.gmask, v, L.gbase);
}

// ---------------------------------------------------------------------------
// OCC
// ---------------------------------------------------------------------------
template <class Work>
__device__ int occ_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, uint32_t attempt,
                           unsigned long long& order_key, uint32_t& crec) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    uint32_t frec = NO_CC;   // this lane's conflicting record
    // read phase: consistent (version, value) pairs into the workspace
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            if (r == NO_CC) {
                S.oldv[j] = Work::load(a, d);
            } else {
                uint64_t* m = a.meta + r;
                // An unlocked version read with acquire, then the value.  The
                // pair is checked later, not here: write keys by the lock CAS
                // (it fails if the version moved), read keys by validation
                // after the commit timestamp.  OCC writers install values only
                // right before publishing a new version, so an unchanged
                // unlocked version proves the value read belongs to it.
                const bool w = Work::writes(d);
                const ulonglong2 opd = w ? a.operands[first + j] : make_ulonglong2(0ull, 0ull);
                for (uint32_t tries = 0;; ++tries) {
                    const uint64_t v1 = ld_acquire(m);
                    if (!(v1 & OCC_LOCK)) {
                        const ulonglong2 v = Work::load(a, d);
                        S.obs[j] = v1;
                        S.oldv[j] = v;
                        if (w) S.newv[j] = Work::compute(a, d, v, opd);
                        break;
                    }
                    if (tries >= a.read_retries) { fail = true; frec = r; break; }
                    __nanosleep(32);
                }
            }
        }
        if (__any_sync(L.gmask, fail)) {
            crec = group_conflict(L, frec);
            return ABORT;
        }
    }
    // lock the write set, no waiting; a changed version fails the CAS too
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops && Work::writes(S.desc[j])) {
            const uint32_t r = Work::rec(a, S.desc[j]);
            bool ok = !collapse_loser(a, r);
            if (ok) ok = (++L.n_atom, cas64(a.meta + r, S.obs[j], S.obs[j] | OCC_LOCK) == S.obs[j]);
            if (ok) held |= 1ull << k; else { fail = true; frec = r; }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        // The commit timestamp is an acquire-release atomic on the clock: its
        // release half orders the write locks before it, its acquire half the
        // validation and the writes after it.  Of two transactions, the one
        // with the later timestamp therefore sees the other's locks: a record
        // it validates that the other locked shows as locked (no write skew,
        // no missed anti-dependency), and timestamp order is a serial order.
        // One lane takes the group's timestamp; the warp barriers around it
        // order the other lanes' locks before it and their reads after it.
        __syncwarp(L.gmask);
        const unsigned long long ts = group_ticket_acq_rel(L, &a.dbs->occ_clock);
        __syncwarp(L.gmask);
        // validate the read set against the versions observed
        for (uint32_t k = 0; k < kmax; ++k) {
            const uint32_t j = L.lig + k * L.G;
            if (j < nops && !Work::writes(S.desc[j])) {
                const uint32_t r = Work::rec(a, S.desc[j]);
                if (r != NO_CC && ld_relaxed(a.meta + r) != S.obs[j]) { fail = true; frec = r; }
            }
        }
        if (!__any_sync(L.gmask, fail)) {
            // write phase, then publish the new version and unlock
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) {
                    const uint32_t j = L.lig + k * L.G;
                    Work::store(a, S.desc[j], S.newv[j], first + j);
                }
            // publish: a release store, so a reader that acquires the new
            // version sees the values written before it
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1)
                    st_release(a.meta + Work::rec(a, S.desc[L.lig + k * L.G]), ts + 1);
            order_key = ts;
            return COMMIT;
        }
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            st_release(a.meta + Work::rec(a, S.desc[j]), S.obs[j]);
        }
    crec = group_conflict(L, frec);
    return ABORT;
}

// ---------------------------------------------------------------------------
// NO_WAIT 2PL
// ---------------------------------------------------------------------------
// With WAIT_DIE, a lock held exclusively by a younger transaction (larger id:
// ids are fixed across restarts) is waited for, within a bound, instead of
// aborting; a younger requester dies as in NO_WAIT.  Waits only ever go from
// older to younger, so they cannot form a cycle.  A lock held shared is not
// waited for (the word does not record the oldest shared holder).
template <class Work, bool WAIT_DIE = false>
__device__ int tpl_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, uint32_t attempt,
                           unsigned long long& order_key, uint32_t& crec) {
    const uint32_t wait_spins = WAIT_DIE ? 256u * (a.read_retries + 1u) : 0u;
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    uint32_t frec = NO_CC;
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            if (r != NO_CC) {
                uint64_t* m = a.meta + r;
                if (!Work::writes(d)) {
                    uint32_t waited = 0;
                    for (uint32_t tries = 0;;) {
                        const uint64_t w = ld_relaxed(m);
                        if (w & TPL_X) {
                            if (WAIT_DIE && t + 1 < (uint32_t)w && waited < wait_spins) {
                                ++waited;
                                __nanosleep(64);
                                continue;
                            }
                            fail = true; frec = r; break;
                        }
                        ++L.n_atom;
                        if (cas64_acquire(m, w, w + TPL_S_ONE) == w) { held |= 1ull << k; break; }
                        if (++tries > a.read_retries) { fail = true; frec = r; break; }
                    }
                } else {
                    bool ok = !collapse_loser(a, r);
                    if (ok) {
                        const uint64_t mine = TPL_X | (uint64_t)(t + 1);
                        ++L.n_atom;
                        uint64_t cur = cas64_acquire(m, 0ull, mine);
                        for (uint32_t waited = 0; WAIT_DIE && cur != 0ull && (cur & TPL_X) &&
                                                  t + 1 < (uint32_t)cur && waited < wait_spins;
                             ++waited) {
                            __nanosleep(64);
                            cur = ld_relaxed(m);
                            if (cur == 0ull) { ++L.n_atom; cur = cas64_acquire(m, 0ull, mine); }
                        }
                        ok = cur == 0ull;
                    }
                    if (ok) held |= 1ull << k; else { fail = true; frec = r; }
                }
            }
            if (!fail) {
                const ulonglong2 v = Work::load(a, d);
                S.oldv[j] = v;
                if (Work::writes(d)) S.newv[j] = Work::compute(a, d, v, a.operands[first + j]);
            }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        // lock point: every lock is held.  The warp barriers order the group's
        // lock acquisitions before the ticket and its releases after it.
        __syncwarp(L.gmask);
        const unsigned long long ts = group_ticket(L, &a.st->ticket);
        __syncwarp(L.gmask);
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                if (Work::writes(S.desc[j])) Work::store(a, S.desc[j], S.newv[j], first + j);
            }
        order_key = ts;
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            uint64_t* m = a.meta + Work::rec(a, S.desc[j]);
            if (!Work::writes(S.desc[j])) { ++L.n_atom; add64_release(m, (uint64_t)0 - TPL_S_ONE); }
            else st_release(m, 0ull);
        }
    if (fail) crec = group_conflict(L, frec);
    return fail ? ABORT : COMMIT;
}

// ---------------------------------------------------------------------------
// basic TO
// ---------------------------------------------------------------------------
template <class Work>
__device__ int to_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                          uint64_t first, uint32_t nops, uint32_t attempt,
                          unsigned long long& order_key, uint32_t& crec) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    const unsigned long long ts = group_ticket(L, &a.dbs->to_clock) + 1;
    ulonglong2* words = reinterpret_cast<ulonglong2*>(a.meta);
    bool fail = false;
    uint32_t frec = NO_CC;
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            if (r == NO_CC) {
                S.oldv[j] = Work::load(a, d);
            } else if (!Work::writes(d)) {
                // read: needs ts > WTS and no uncommitted write, then RTS =
                // max(RTS, ts).  RTS only grows, so a 64-bit atomicMax raises it
                // without failing; the WTS half read unchanged before the value
                // and after the raise proves the value belongs to that WTS, and
                // a writer's 128-bit CAS fails once RTS moved.
                ulonglong2* m = words + r;
                uint64_t* wts_word = reinterpret_cast<uint64_t*>(&m->y);
                uint64_t* rts_word = reinterpret_cast<uint64_t*>(&m->x);
                for (uint32_t tries = 0;; ++tries) {
                    const uint64_t y1 = ld_acquire(wts_word);
                    if ((y1 & TO_DIRTY) || ts < y1) { fail = true; frec = r; break; }
                    // raising RTS early only turns away older writers sooner, so
                    // it goes out together with the value load
                    max64(rts_word, ts);
                    ++L.n_atom;
                    const ulonglong2 v = Work::load(a, d);
                    fence_acq_rel();
                    if (ld_relaxed(wts_word) == y1) { S.oldv[j] = v; break; }
                    if (tries >= a.read_retries) { fail = true; frec = r; break; }
                }
            } else {
                // write: needs ts > RTS and ts > WTS; mark dirty with WTS = ts.
                // The value is read before the mark, after the word (with
                // acquire): values change only while a word is dirty, and a
                // writer that marked it since changed the word, so the value
                // belongs to w if the CAS from w succeeds -- the load then lies
                // outside the record's tenure.
                ulonglong2* m = words + r;
                bool ok = !collapse_loser(a, r);
                ulonglong2 v = make_ulonglong2(0ull, 0ull);
                for (uint32_t tries = 0; ok; ++tries) {
                    const ulonglong2 w = ld128_acquire(m);
                    if ((w.y & TO_DIRTY) || ts < w.x || ts < w.y) { ok = false; break; }
                    v = Work::load(a, d);
                    ++L.n_atom;
                    const ulonglong2 o = cas128_acquire(m, w, make_ulonglong2(w.x, TO_DIRTY | ts));
                    if (o.x == w.x && o.y == w.y) { S.obs[j] = w.y; break; }
                    if (tries >= a.read_retries) { ok = false; break; }
                }
                if (ok) {
                    held |= 1ull << k;
                    S.oldv[j] = v;
                    S.newv[j] = Work::compute(a, d, v, a.operands[first + j]);
                } else {
                    fail = true;
                    frec = r;
                }
            }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    // While dirty, nobody else changes a word, so only its WTS half is
    // rewritten: the new WTS at commit, the saved one on abort.
    if (!fail) {
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                Work::store(a, S.desc[j], S.newv[j], first + j);
            }
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1)
                st_release(reinterpret_cast<uint64_t*>(&words[Work::rec(a, S.desc[L.lig + k * L.G])].y), ts);
        order_key = ts;
        return COMMIT;
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            st_release(reinterpret_cast<uint64_t*>(&words[Work::rec(a, S.desc[j])].y), S.obs[j]);
        }
    crec = group_conflict(L, frec);
    return ABORT;
}

// ---------------------------------------------------------------------------
// TicToc
// ---------------------------------------------------------------------------
// Maximum of a 64-bit value over the lanes of a group (groups are aligned
// power-of-two sub-warps, so xor shuffles stay inside the group).
__device__ __forceinline__ uint64_t group_max64(const Lane& L, uint64_t v) {
    for (uint32_t off = L.G >> 1; off > 0; off >>= 1) {
        const uint64_t o = __shfl_xor_sync(L.gmask, v, off);
        v = o > v ? o : v;
    }
    return v;
}

// Read phase as OCC's, recording each record's wts and rts; the write set is
// locked without waiting, each lock a 128-bit CAS that also fixes the rts it
// locks at (when only the rts moved since the read, a reader extended it: the
// lock is retried at the new rts); the commit timestamp is computed, not drawn
// from a clock: at least every record read's wts and one past every record
// written's rts.  A record read whose observed rts already covers the timestamp needs
// no check; otherwise its rts is extended to the timestamp with a 128-bit CAS
// that also proves the version unchanged and unlocked.  Writes publish
// wts = rts = timestamp.  Two commits never tie on a timestamp when they
// conflict on a write-write or read-then-overwrite pair; the only tie is a
// reader of a version at that version's own timestamp, and the writer's
// sequence number, taken before it publishes, orders it first.  The serial
// order is (timestamp, sequence number).
template <class Work>
__device__ int tictoc_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                              uint64_t first, uint32_t nops, uint32_t attempt,
                              unsigned long long& order_key, uint32_t& seq_out, uint32_t& crec) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    ulonglong2* words = reinterpret_cast<ulonglong2*>(a.meta);
    bool fail = false;
    uint32_t frec = NO_CC;
    // read phase: (wts, value, rts) of one version.  A read whose rts already
    // covers the commit timestamp is not checked again, so the three must be
    // one snapshot: wts is read again after the value and rts, and the read
    // retried if a writer locked or published in between.
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            if (r == NO_CC) {
                S.oldv[j] = Work::load(a, d);
            } else {
                ulonglong2* m = words + r;
                uint64_t* wts_word = reinterpret_cast<uint64_t*>(&m->y);
                uint64_t* rts_word = reinterpret_cast<uint64_t*>(&m->x);
                const bool w = Work::writes(d);
                const ulonglong2 opd = w ? a.operands[first + j] : make_ulonglong2(0ull, 0ull);
                for (uint32_t tries = 0;; ++tries) {
                    const uint64_t y1 = ld_acquire(wts_word);
                    if (!(y1 & TT_LOCK)) {
                        const ulonglong2 v = Work::load(a, d);
                        const uint64_t rts = ld_relaxed(rts_word);
                        fence_acq_rel();
                        if (ld_relaxed(wts_word) == y1) {
                            S.obs[j] = y1;
                            S.oldv[j] = v;
                            S.aux[j] = rts;
                            if (w) S.newv[j] = Work::compute(a, d, v, opd);
                            break;
                        }
                    }
                    if (tries >= a.read_retries) { fail = true; frec = r; break; }
                    __nanosleep(32);
                }
            }
        }
        if (__any_sync(L.gmask, fail)) {
            crec = group_conflict(L, frec);
            return ABORT;
        }
    }
    // lock the write set, no waiting; a changed wts fails the CAS too
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops && Work::writes(S.desc[j])) {
            const uint32_t r = Work::rec(a, S.desc[j]);
            bool ok = !collapse_loser(a, r);
            if (ok) {
                ulonglong2 expect = make_ulonglong2(S.aux[j], S.obs[j]);
                ok = false;
                for (uint32_t tries = 0; tries <= a.read_retries; ++tries) {
                    ++L.n_atom;
                    const ulonglong2 o = cas128_acquire(words + r, expect,
                                                        make_ulonglong2(expect.x, expect.y | TT_LOCK));
                    if (o.x == expect.x && o.y == expect.y) { ok = true; break; }
                    if (o.y != S.obs[j]) break;          // written or locked since
                    expect.x = o.x;
                }
                if (ok) S.aux[j] = expect.x;             // rts under the lock
            }
            if (ok) held |= 1ull << k; else { fail = true; frec = r; }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        // the timestamp: a locked record's rts no longer moves (extensions
        // need it unlocked), and the lock fixed it
        uint64_t c = 0;
        for (uint32_t k = 0; k < kmax; ++k) {
            const uint32_t j = L.lig + k * L.G;
            if (j < nops) {
                const uint32_t r = Work::rec(a, S.desc[j]);
                if (r == NO_CC) continue;
                const uint64_t cand = Work::writes(S.desc[j]) ? S.aux[j] + 1 : S.obs[j];
                c = cand > c ? cand : c;
            }
        }
        const uint64_t ts = group_max64(L, c);
        // the sequence number goes out together with the validation
        __syncwarp(L.gmask);
        unsigned long long sq = 0;
        if (L.lig == 0) sq = agg_ticket_acq_rel(&a.st->ticket, &L.n_atom);
        // validate the read set at the timestamp, extending rts where needed
        for (uint32_t k = 0; k < kmax; ++k) {
            const uint32_t j = L.lig + k * L.G;
            if (j < nops && !Work::writes(S.desc[j])) {
                const uint32_t r = Work::rec(a, S.desc[j]);
                if (r == NO_CC || S.aux[j] >= ts) continue;
                ulonglong2* m = words + r;
                bool ok = false;
                for (uint32_t tries = 0; tries <= a.read_retries; ++tries) {
                    const ulonglong2 w = ld_slot16(m);
                    if (w.y != S.obs[j]) break;                  // written or locked since
                    if (w.x >= ts) { ok = true; break; }
                    ++L.n_atom;
                    const ulonglong2 o = cas128(m, w, make_ulonglong2(ts, w.y));
                    if (o.x == w.x && o.y == w.y) { ok = true; break; }
                }
                if (!ok) { fail = true; frec = r; }
            }
        }
        sq = __shfl_sync(L.gmask, sq, L.gbase);
        __syncwarp(L.gmask);
        if (!__any_sync(L.gmask, fail)) {
            // write phase, then publish the version [ts, ts] and unlock
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) {
                    const uint32_t j = L.lig + k * L.G;
                    Work::store(a, S.desc[j], S.newv[j], first + j);
                    ulonglong2* m = words + Work::rec(a, S.desc[j]);
                    st_relaxed(reinterpret_cast<uint64_t*>(&m->x), ts);
                    st_release(reinterpret_cast<uint64_t*>(&m->y), ts);
                }
            order_key = ts;
            seq_out = (uint32_t)sq;
            return COMMIT;
        }
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            st_release(reinterpret_cast<uint64_t*>(&words[Work::rec(a, S.desc[j])].y), S.obs[j]);
        }
    crec = group_conflict(L, frec);
    return ABORT;
}

// ---------------------------------------------------------------------------
// MVCC (multi-version TO)
// ---------------------------------------------------------------------------
// The multi-version form of basic TO (Sec. II, "Multi-version Concurrency
// Control"; Sec. III-E, "MVCC"): every write makes a new immutable version
// stamped with its writer's timestamp, and a read returns the version whose
// validity interval holds its timestamp -- the newest version older than it.
// As in the paper, the latest versions have one array (a version pointer per
// (record, field) slot) and the history another (the batch's version store:
// entries taken from one counter, as many as the batch's committed writes, so
// n_ops entries always suffice, each linked to its slot's previous entry);
// the table slot is every slot's oldest version and is not written until the
// batch ends (launch_mv_flatten).  Concurrency control is per record, in the
// record's head word (engine.cuh): newest version's wts and rts, and a
// pending writer.
//  * Write at ts: needs no pending writer, wts < ts and rts <= ts; reads its
//    slot's newest version (the pointer's entry, or the table slot) and then
//    installs itself as the pending writer by a CAS from the head it read:
//    if the CAS succeeds, no writer became pending or committed since that
//    head, so the version read is still the newest, and none can add one
//    while it is pending.
//  * Read at ts: aborts if an older writer is pending (its version might be
//    the one to read); if the record's newest version is older than ts it
//    raises the head's rts to ts by a CAS, so that no writer older than ts can
//    add a version under it; it then walks its slot's entries from the newest
//    to the first older than ts (newer ones, from writers after ts, are
//    stepped over), or takes the table slot.
//  * Commit: the new entries go into the store (a range of it taken once per
//    transaction, before its first attempt), then (release) the slots'
//    version pointers, then (release) each head is set to (ts, ts, no writer)
//    by a CAS loop that starts from the head this writer installed -- only
//    readers' rts raises, all below ts, can move it meanwhile.  Abort: the
//    pending marks are withdrawn the same way.
// Versions are stored when the writer commits, so an aborted attempt leaves
// nothing to undo but its pending marks (the paper's version pointers are
// likewise updated at commit).  Commit order: the timestamp, batch-relative
// 32-bit (a batch that would exceed 2^32 - 1 timestamps ends
// GCC_DEVERR_TS_OVERFLOW).  The protocol was checked against serial replay on
// interleavings before the kernel existed.
constexpr uint32_t MV_WALK_MAX = 1u << 16;   // entries a read may step over

__device__ __forceinline__ uint32_t* mv_slot_ptr(const ExecArgs& a, uint64_t d) {
    return a.mv_slot + (uint64_t)op_field(d) * a.n_records + op_key(d);
}

__device__ __forceinline__ uint32_t mv_pointer(const ExecArgs& a, uint64_t d) {
    uint32_t e;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(e) : "l"(mv_slot_ptr(a, d)) : "memory");
    return e;
}

// The newest version of op d's slot older than ts: its entries from the
// newest (version pointer e, read with acquire) down, else the table slot.
// An entry's value is loaded beside its timestamp.  False when the walk would
// step over more than MV_WALK_MAX entries (the attempt then aborts).
template <class Work>
__device__ __forceinline__ bool mv_version(const ExecArgs& a, uint64_t d, uint32_t ts, uint32_t e,
                                           ulonglong2& out) {
    for (uint32_t n = 0; e != 0; ++n) {
        if (n >= MV_WALK_MAX) return false;
        const uint32_t i = e - 1;
        const uint32_t wts = ld_relaxed_u32(a.mv_wts + i);
        const uint32_t nxt = ld_relaxed_u32(a.mv_next + i);
        const ulonglong2 v = ld_slot16(a.mv_val + i);
        if (wts < ts) {
            out = v;
            return true;
        }
        e = nxt;
    }
    out = Work::load(a, d);
    return true;
}

// Withdraw a pending mark (abort) or publish a committed version: a CAS loop
// that keeps whatever rts raises happened meanwhile.  Only readers move the
// word while this transaction's mark is on it, each raise at most once per
// reader attempt, so the loop ends; it is bounded all the same, and a word
// still not updated after 2^24 tries sets GCC_DEVERR_DEADLINE.
__device__ __forceinline__ void mv_set_head(const ExecArgs& a, ulonglong2* m, bool commit,
                                            uint32_t ts, uint64_t installed, uint32_t& n_atom) {
    // first guess: the head as this writer installed it (wts|rts, pending ts)
    ulonglong2 cur = make_ulonglong2(installed, mv_pack(ts, 0u));
    for (uint32_t tries = 0;; ++tries) {
        if (tries >= (1u << 24)) {
            atomicOr(&a.st->error, GCC_DEVERR_DEADLINE);
            return;
        }
        ulonglong2 nw;
        if (commit) {
            const uint32_t rts = mv_hi(cur.x) > ts ? mv_hi(cur.x) : ts;
            nw = make_ulonglong2(mv_pack(ts, rts), 0ull);
        } else {
            nw = make_ulonglong2(cur.x, mv_pack(0u, mv_hi(cur.y)));
        }
        ++n_atom;
        const ulonglong2 o = cas128(m, cur, nw);
        if (o.x == cur.x && o.y == cur.y) return;
        cur = o;
    }
}

// The transaction's range of the version store, taken once before its first
// attempt: lane i's write ops take the entries after those of the lanes
// before it.  Returns the lane's first entry.
template <class Work>
__device__ __forceinline__ uint32_t mv_entries(const ExecArgs& a, const Lane& L, const Stage& S,
                                               uint32_t nops, uint32_t& base) {
    uint32_t mine = 0;
    for (uint32_t j = L.lig; j < nops; j += L.G) mine += Work::writes(S.desc[j]) ? 1u : 0u;
    uint32_t incl = mine;                                   // inclusive scan over the group
    for (uint32_t off = 1; off < L.G; off <<= 1) {
        const uint32_t v = __shfl_up_sync(L.gmask, incl, off, L.G);
        if (L.lig >= off) incl += v;
    }
    if (base == NO_CC) {
        const uint32_t total = __shfl_sync(L.gmask, incl, L.gbase + L.G - 1);
        unsigned long long b = 0;
        if (L.lig == 0 && total) { b = atomicAdd(&a.st->mv_used, (unsigned long long)total); ++L.n_atom; }
        base = (uint32_t)__shfl_sync(L.gmask, b, L.gbase);
    }
    return base + incl - mine;
}

template <class Work>
__device__ int mvcc_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                            uint64_t first, uint32_t nops, uint32_t attempt,
                            unsigned long long& order_key, uint32_t& crec, uint32_t& mv_base) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    uint32_t e = mv_entries<Work>(a, L, S, nops, mv_base);
    const unsigned long long t64 = group_ticket(L, &a.st->ticket) + 1;
    if (t64 >= 0xFFFFFFFFull) {
        if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_TS_OVERFLOW);
        return GIVE_UP;
    }
    const uint32_t ts = (uint32_t)t64;
    ulonglong2* heads = reinterpret_cast<ulonglong2*>(a.meta);
    bool fail = false;
    uint32_t frec = NO_CC;
    uint64_t held = 0;               // ops whose record this attempt marked pending
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            ulonglong2* m = heads + r;
            if (!Work::writes(d)) {
                bool ok = false;
                for (uint32_t tries = 0; tries <= a.read_retries; ++tries) {
                    const ulonglong2 h = ld128_acquire(m);
                    const uint32_t wts = mv_lo(h.x), rts = mv_hi(h.x), pend = mv_lo(h.y);
                    if (pend != 0 && pend < ts) break;          // an older writer is pending
                    // the version pointer beside the rts raise: if the CAS
                    // from h succeeds, no version older than ts was added
                    // after h (its writer would have changed the head first)
                    const uint32_t pe = mv_pointer(a, d);
                    if (wts < ts && rts < ts) {
                        ++L.n_atom;
                        const ulonglong2 o = cas128_acquire(m, h, make_ulonglong2(mv_pack(wts, ts), h.y));
                        if (o.x != h.x || o.y != h.y) continue;
                    }
                    ok = mv_version<Work>(a, d, ts, pe, S.oldv[j]);
                    break;
                }
                if (!ok) { fail = true; frec = r; }
            } else {
                bool ok = !collapse_loser(a, r);
                for (uint32_t tries = 0; ok && tries <= a.read_retries; ++tries) {
                    const ulonglong2 h = ld128_acquire(m);
                    const uint32_t wts = mv_lo(h.x), rts = mv_hi(h.x), pend = mv_lo(h.y);
                    if (pend != 0 || wts >= ts || rts > ts) { ok = false; break; }
                    // the slot's newest version, before the pending mark: its
                    // pointer's entry or the table slot (every committed
                    // version is older than ts); still the newest if the CAS
                    // from h succeeds
                    uint32_t pe;
                    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(pe) : "l"(mv_slot_ptr(a, d)) : "memory");
                    const ulonglong2 v = pe ? ld_slot16(a.mv_val + (pe - 1)) : Work::load(a, d);
                    ++L.n_atom;
                    const ulonglong2 o = cas128_acquire(m, h, make_ulonglong2(h.x, mv_pack(ts, mv_hi(h.y))));
                    if (o.x != h.x || o.y != h.y) {
                        if (tries == a.read_retries) ok = false;
                        continue;
                    }
                    held |= 1ull << k;
                    S.obs[j] = pe;                              // the entry it supersedes
                    S.aux[j] = h.x;                             // the head's first word as installed
                    S.oldv[j] = v;
                    S.newv[j] = Work::compute(a, d, v, a.operands[first + j]);
                    break;
                }
                if (!ok) { fail = true; frec = r; }
            }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        // every write op holds its record now: the lane's entries, in op order
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                const uint64_t d = S.desc[j];
                a.mv_wts[e] = ts;
                a.mv_next[e] = (uint32_t)S.obs[j];
                a.mv_rec[e] = Work::rec(a, d);
                a.mv_field[e] = op_field(d);
                st_slot16(a.mv_val + e, S.newv[j]);
                S.obs[j] = e + 1;                               // the entry it publishes
                ++e;
            }
        if (held) {
            // the entries before the version pointers that name them, and
            // the pointers before the heads that admit readers above ts
            fence_acq_rel();
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) {
                    const uint32_t j = L.lig + k * L.G;
                    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;"
                                 ::"l"(mv_slot_ptr(a, S.desc[j])), "r"((uint32_t)S.obs[j]) : "memory");
                }
            fence_acq_rel();
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) {
                    const uint32_t j = L.lig + k * L.G;
                    mv_set_head(a, heads + Work::rec(a, S.desc[j]), true, ts, S.aux[j], L.n_atom);
                }
        }
        order_key = ts;
        return COMMIT;
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            mv_set_head(a, heads + Work::rec(a, S.desc[j]), false, ts, S.aux[j], L.n_atom);
        }
    crec = group_conflict(L, frec);
    return ABORT;
}

// ---------------------------------------------------------------------------
// DET
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool det_wait(const ExecArgs& a, uint64_t* m, bool is_write,
                                         uint32_t need) {
    uint64_t t_begin = 0;
    for (uint32_t spins = 0;; ++spins) {
        const uint64_t c = ld_acquire(m);
        const uint32_t done = is_write ? (uint32_t)(c >> 32) : (uint32_t)c;
        if (done >= need) return true;
        if ((spins & 31) == 31) {
            const uint64_t now = globaltimer();
            if (t_begin == 0) t_begin = now;
            else if (now - t_begin > a.wait_budget_ns) {
                atomicOr(&a.st->error, GCC_DEVERR_WAIT_BUDGET);
                return false;
            }
            if (*reinterpret_cast<volatile unsigned*>(&a.st->error) &
                (GCC_DEVERR_WAIT_BUDGET | GCC_DEVERR_DEADLINE))
                return false;
            __nanosleep(64);
        }
    }
}

template <class Work>
__device__ int det_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, unsigned long long& order_key) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    for (uint32_t k = 0; k < kmax && !fail; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            const uint32_t r = Work::rec(a, d);
            if (r == NO_CC) {
                S.oldv[j] = Work::load(a, d);
                continue;
            }
            uint64_t* m = a.meta + r;
            const bool w = Work::writes(d);
            if (!det_wait(a, m, w || a.det_all, a.need[first + j])) { fail = true; break; }
            const ulonglong2 v = Work::load(a, d);
            S.oldv[j] = v;
            if (w) Work::store(a, d, Work::compute(a, d, v, a.operands[first + j]), first + j);
            add64_release(m, w ? DET_WRITE_DONE : DET_READ_DONE);
            ++L.n_atom;
        }
    }
    if (__any_sync(L.gmask, fail)) return GIVE_UP;
    order_key = t;
    return COMMIT;
}

// An invalid transaction never runs, but its accesses are in the batch's
// access table: advance its records' counters in order so that later
// transactions on those records are not held up.
template <class Work>
__device__ void det_skip(const ExecArgs& a, const Lane& L, uint64_t first, uint32_t nops) {
    if (first + nops > a.n_ops) return;
    for (uint32_t j = L.lig; j < nops; j += L.G) {
        const uint64_t d = a.ops[first + j];
        const uint32_t rec = cc_record(d, Work::SCHEMA, a.n_warehouses, NO_CC);
        if (rec >= a.n_meta) continue;
        const bool w = kind_writes(op_kind(d));
        if (det_wait(a, a.meta + rec, w || a.det_all, a.need[first + j])) {
            add64(a.meta + rec, w ? DET_WRITE_DONE : DET_READ_DONE);
            ++L.n_atom;
        }
    }
}

// Nanoseconds an aborted transaction sits out: backoff_base_ns times a number
// uniform in [0, window], the window doubling with each abort up to
// backoff_cap_ns / backoff_base_ns.  Waits are deadlines on the global timer,
// not round counts: a round lasts a few hundred nanoseconds in an idle warp
// and several microseconds in a busy one.
__device__ __forceinline__ uint64_t backoff_ns(const ExecArgs& a, uint32_t t, uint32_t attempts) {
    if (a.backoff_base_ns == 0) return 0;
    uint64_t cap = a.backoff_cap_ns / a.backoff_base_ns;
    if (cap < 1) cap = 1;
    const uint32_t sh = attempts - 1 < 20 ? attempts - 1 : 20;
    uint64_t window = 1ull << sh;
    if (window > cap) window = cap;
    return (mix64(a.seed ^ ((uint64_t)t << 24) ^ attempts) % (window + 1)) * a.backoff_base_ns;
}

// Retry queues.  A transaction that has aborted queue_after times or more and
// conflicted on a record backs off as above, then takes a ticket in the FIFO
// queue that record hashes to and re-attempts when the queue admits its
// ticket; it holds nothing while it waits, so the schemes'
// attempts stay exactly as described above (no attempt ever waits for a
// lock).  A queue admits the oldest `queue_width` unfinished tickets; an
// admitted transaction counts its ticket finished when its attempt ends.  At
// low contention a queue holds one transaction, which re-attempts at once;
// on a hot record the aborted transactions re-attempt a few at a time instead
// of all together.  A queue word is (tickets taken << 32) | tickets finished.
// Admitted transactions always finish their attempt, so a queue never stalls;
// a transaction still waiting at the kernel deadline gives up and abandons its
// ticket, and the words are zeroed before every batch.
constexpr uint32_t NO_Q = 0xffffffffu;

__device__ __forceinline__ uint32_t queue_of(const ExecArgs& a, uint32_t rec) {
    return (uint32_t)mix64(rec) & a.rq_mask;
}

// Nanoseconds a waiter sleeps before looking again, `ahead` turns from its
// own: about one estimated turn per transaction ahead, so a queue word is
// read a few times per turn however long the queue.
__device__ __forceinline__ uint64_t queue_wait_ns(const ExecArgs& a, uint32_t ahead) {
    const uint64_t w = (uint64_t)(ahead - 1) * a.queue_turn_ns;
    return w < a.backoff_cap_ns ? w : a.backoff_cap_ns;
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
struct Counters {
    unsigned commits = 0, aborts = 0, timeouts = 0, invalid = 0, max_att = 0, atomics = 0;
};

// Hands out transactions of one batch in id order.
// Transactions are handed out in chunks of CHUNK consecutive ids per lane
// group: one atomic per warp and chunk on the shared counter instead of one
// per transaction.  The deterministic scheme's waits need every fetched
// transaction to be running (a group must never hold an unstarted id that
// another group waits on while the warp's round waits for that group), so it
// fetches one id at a time.
template <unsigned CHUNK>
struct SingleFetch {
    const ExecArgs* a;
    unsigned long long next_id = 0, end_id = 0;
    __device__ __forceinline__ bool next(const Lane& L, uint32_t& t, const ExecArgs*& A) {
        if (next_id >= end_id) {
            unsigned long long tt = 0;
            if (L.lig == 0) tt = agg_ticket(&a->st->fetch, CHUNK, &L.n_atom);
            next_id = __shfl_sync(L.gmask, tt, L.gbase);
            end_id = next_id + CHUNK;
        }
        if (next_id >= a->n_txns) return false;
        t = (uint32_t)next_id++;
        A = a;
        return true;
    }
    __device__ __forceinline__ void done(const Lane&, const ExecArgs&, Counters&) {}
};

// The execution loop of one lane group: take a transaction, stage and check
// it, attempt it round after round until it commits or gives up.
template <int SCHEME, class Work, class Fetch>
__device__ void group_loop(Fetch& F, const Lane& L, const Stage& S, uint32_t M, uint64_t deadline,
                           Counters& c) {
    constexpr bool DENSE =
        SCHEME == GCC_NO_WAIT_2PL || SCHEME == GCC_2PL_WAIT_DIE || SCHEME == GCC_DET;
    bool finished = false, has = false, served = false;
    bool skip = false;            // DET: an invalid transaction's accesses still to advance
    uint32_t t = 0, nops = 0, attempts = 0;
    uint64_t wake = 0;            // global-timer time before which the group waits
    uint32_t qi = NO_Q, qt = 0;   // retry queue and ticket while queued
    uint32_t pq = NO_Q;           // queue to join once the backoff is over
    uint32_t mv_base = NO_CC;     // MVCC: the transaction's version-store range
    uint64_t first = 0;
    const ExecArgs* A = nullptr;

    for (;;) {
        // 1. groups without a transaction take the next one
        if (!has && !finished) {
            if (!F.next(L, t, A)) {
                finished = true;
            } else {
                const ExecArgs& a = *A;
                const gcc_txn tx = a.txns[t];
                nops = tx.n_ops;
                first = tx.first_op;
                bool bad = nops > M || !Work::valid_txn(a, tx) || first + nops > a.n_ops;
                if (!bad) {
                    for (uint32_t j = L.lig; j < nops; j += L.G) {
                        const uint64_t d = a.ops[first + j];
                        S.desc[j] = d;
                        if (!Work::valid_op(a, d)) bad = true;
                    }
                }
                __syncwarp(L.gmask);
                if (!__any_sync(L.gmask, bad)) {
                    // keys of one transaction must be distinct records
                    for (uint32_t j = L.lig; j < nops; j += L.G) {
                        const uint32_t rj = Work::rec(a, S.desc[j]);
                        if (rj == NO_CC) continue;
                        for (uint32_t i = 0; i < j; ++i)
                            if (Work::rec(a, S.desc[i]) == rj) bad = true;
                    }
                    bad = bad || !Work::valid_shape(a, S, nops, tx.type);
                }
                if (__any_sync(L.gmask, bad)) {
                    if (L.lig == 0) {
                        a.results[t] = gcc_txn_result{GCC_TXN_INVALID, 0u, ~0ull};
                        if (!DENSE) a.order_key[t] = ~0ull;
                        atomicOr(&a.st->error, GCC_DEVERR_INVALID);
                        ++c.invalid;
                    }
                    if constexpr (SCHEME == GCC_DET) {
                        // its accesses advance their records' counters in the
                        // attempt step, where the groups they wait for run:
                        // waiting here, before the warp-wide vote below,
                        // would hold up a predecessor in the same warp
                        has = true;
                        skip = true;
                        attempts = 0;
                        wake = 0;
                    } else {
                        F.done(L, a, c);
                    }
                } else {
                    has = true;
                    attempts = 0;
                    wake = 0;
                    mv_base = NO_CC;
                }
                __syncwarp(L.gmask);
            }
        }
        if (__all_sync(0xffffffffu, finished)) break;

        // 2. one attempt per group holding a transaction that is neither
        // backing off nor waiting for its turn in a retry queue
        bool go = false, expired = false;
        // Every decision below must be the same on all lanes of a group (they
        // meet in group-wide shuffles and votes), so a group reads the timer
        // once, on its base lane.
        const uint64_t now = __shfl_sync(0xffffffffu, globaltimer(), L.gbase);
        if (has && now < wake) {
            // backing off, or not yet due to look at its queue
        } else if (has && (pq != NO_Q || (qi != NO_Q && !served))) {
            const ExecArgs& a = *A;
            uint64_t w = 0;
            if (pq != NO_Q) {
                // the backoff is over: take a ticket; the word before it
                // also tells how many tickets have finished
                qi = pq;
                pq = NO_Q;
                if (L.lig == 0) { w = add64(a.rq + qi, 1ull << 32); ++L.n_atom; }
                w = __shfl_sync(L.gmask, w, L.gbase);
                qt = (uint32_t)(w >> 32);
            } else {
                if (L.lig == 0) w = ld_relaxed(a.rq + qi);
                w = __shfl_sync(L.gmask, w, L.gbase);
            }
            // tickets taken before ours minus tickets finished; negative once
            // later tickets finished first (queue_width > 1)
            const int32_t ahead = (int32_t)(qt - (uint32_t)w);
            if (ahead < (int32_t)a.queue_width) {
                served = go = true;
            } else if (now > deadline) {
                expired = true;                // the ticket is abandoned
                qi = NO_Q;
            } else {
                wake = now + queue_wait_ns(a, (uint32_t)(ahead - (int32_t)a.queue_width + 1));
            }
        } else if (has) {
            go = true;
        }
        if (go || expired) {
            const ExecArgs& a = *A;
            unsigned long long order_key = 0;
            uint32_t crec = NO_CC, seq = 0;
            int outcome = GIVE_UP;
            if (go && skip) {
                det_skip<Work>(a, L, first, nops);
                outcome = SKIPPED;
            } else if (go) {
                ++attempts;
                if constexpr (SCHEME == GCC_OCC)
                    outcome = occ_attempt<Work>(a, L, S, t, first, nops, attempts, order_key, crec);
                else if constexpr (SCHEME == GCC_NO_WAIT_2PL)
                    outcome = tpl_attempt<Work>(a, L, S, t, first, nops, attempts, order_key, crec);
                else if constexpr (SCHEME == GCC_TO)
                    outcome = to_attempt<Work>(a, L, S, t, first, nops, attempts, order_key, crec);
                else if constexpr (SCHEME == GCC_2PL_WAIT_DIE)
                    outcome = tpl_attempt<Work, true>(a, L, S, t, first, nops, attempts, order_key,
                                                      crec);
                else if constexpr (SCHEME == GCC_TICTOC)
                    outcome = tictoc_attempt<Work>(a, L, S, t, first, nops, attempts, order_key,
                                                   seq, crec);
                else if constexpr (SCHEME == GCC_MVCC)
                    outcome = mvcc_attempt<Work>(a, L, S, t, first, nops, attempts, order_key,
                                                 crec, mv_base);
                else
                    outcome = det_attempt<Work>(a, L, S, t, first, nops, order_key);
            } else if (L.lig == 0) {
                atomicOr(&a.st->error, GCC_DEVERR_DEADLINE);
            }
            if (served) {                      // pass the queue's turn on
                if (L.lig == 0) { add64(a.rq + qi, 1ull); ++L.n_atom; }
                served = false;
                qi = NO_Q;
            }
            if (outcome == ABORT) {
                if (L.lig == 0) ++c.aborts;
                const uint64_t t2 = __shfl_sync(L.gmask, globaltimer(), L.gbase);
                if (attempts >= a.max_attempts) {
                    if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_ATTEMPTS);
                    outcome = GIVE_UP;
                } else if (t2 > deadline) {
                    if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_DEADLINE);
                    outcome = GIVE_UP;
                } else {
                    // randomized backoff first (it breaks the symmetry of two
                    // transactions that keep aborting each other), then the
                    // queue of the record it conflicted on
                    wake = t2 + backoff_ns(a, t, attempts);
                    if (a.rq && crec != NO_CC && attempts >= a.queue_after)
                        pq = queue_of(a, crec);
                }
            }
            if (outcome == COMMIT) {
                for (uint32_t j = L.lig; j < nops; j += L.G) a.reads[first + j] = S.oldv[j];
                Work::commit_step(a, L, S, t, first, nops);
                if (L.lig == 0) {
                    // 2PL tickets are dense already; OCC/TO keys are densified later
                    a.results[t] = gcc_txn_result{GCC_TXN_COMMITTED, attempts,
                                                  DENSE ? (uint64_t)order_key : ~0ull};
                    if (!DENSE) a.order_key[t] = order_key;
                    if constexpr (SCHEME == GCC_TICTOC) a.seq[t] = seq;
                    ++c.commits;
                }
            } else if (outcome == GIVE_UP) {
                if (L.lig == 0) {
                    a.results[t] = gcc_txn_result{GCC_TXN_TIMEOUT, attempts, ~0ull};
                    if (!DENSE) a.order_key[t] = ~0ull;
                    ++c.timeouts;
                }
            }
            if (outcome != ABORT) {
                if (L.lig == 0 && attempts > c.max_att) c.max_att = attempts;
                has = false;
                skip = false;
                F.done(L, a, c);
            }
            __syncwarp(L.gmask);
        }
        // 3. a warp where nobody attempted this round sleeps until its
        // earliest wake-up (32 ns .. 1 us)
        if (!__any_sync(0xffffffffu, go)) {
            const uint64_t t1 = globaltimer();
            uint32_t rel = 1000;
            if (has && wake > t1) rel = wake - t1 < 1000 ? (uint32_t)(wake - t1) : 1000u;
            else if (has || !finished) rel = 32;   // due now, or about to fetch
            rel = __reduce_min_sync(0xffffffffu, rel);
            __nanosleep(rel < 32 ? 32 : rel);
        }
    }
}

// Lane-group geometry and shared-memory staging of one block.
__device__ __forceinline__ void setup_lanes(uint32_t G, uint32_t M, Lane& L, Stage& S) {
    extern __shared__ __align__(16) unsigned char smem[];
    L.G = G;
    L.lane = threadIdx.x & 31;
    L.lig = L.lane & (L.G - 1);
    L.gbase = L.lane & ~(L.G - 1);
    L.gmask = (L.G == 32) ? 0xffffffffu : (((1u << L.G) - 1u) << L.gbase);
    const uint32_t slots = blockDim.x / L.G;
    const uint32_t slot = threadIdx.x / L.G;
    uint64_t* w64 = reinterpret_cast<uint64_t*>(smem);
    S.desc = w64 + (size_t)slot * M;
    S.obs = w64 + (size_t)slots * M + (size_t)slot * M;
    ulonglong2* w128 = reinterpret_cast<ulonglong2*>(w64 + 2 * (size_t)slots * M);
    S.oldv = w128 + (size_t)slot * M;
    S.newv = w128 + (size_t)slots * M + (size_t)slot * M;
    S.aux = reinterpret_cast<uint64_t*>(w128 + 2 * (size_t)slots * M) + (size_t)slot * M;
}

// Warp-reduced counters into a batch's state: one atomic per warp and field.
__device__ __forceinline__ void flush_counters(BatchState* st, Counters& c) {
    const unsigned commits = __reduce_add_sync(0xffffffffu, c.commits);
    const unsigned aborts = __reduce_add_sync(0xffffffffu, c.aborts);
    const unsigned timeouts = __reduce_add_sync(0xffffffffu, c.timeouts);
    const unsigned invalid = __reduce_add_sync(0xffffffffu, c.invalid);
    const unsigned max_att = __reduce_max_sync(0xffffffffu, c.max_att);
    const unsigned atoms = __reduce_add_sync(0xffffffffu, c.atomics);
    if ((threadIdx.x & 31) == 0) {
        if (atoms) atomicAdd(&st->atomics, (unsigned long long)atoms);
        if (commits) atomicAdd(&st->committed, (unsigned long long)commits);
        if (aborts) atomicAdd(&st->aborts, (unsigned long long)aborts);
        if (timeouts) atomicAdd(&st->timeouts, (unsigned long long)timeouts);
        if (invalid) atomicAdd(&st->invalid, (unsigned long long)invalid);
        if (max_att) atomicMax(&st->max_attempts, (unsigned long long)max_att);
    }
}

template <int SCHEME, class Work>
__global__ void __launch_bounds__(1024) exec_kernel(const __grid_constant__ ExecArgs a) {
    Lane L;
    Stage S;
    setup_lanes(a.lanes, a.max_ops, L, S);
    // one deadline per warp: lanes must agree on every time comparison
    const uint64_t deadline = __shfl_sync(0xffffffffu, globaltimer(), 0) + a.deadline_ns;
    Counters c;
    SingleFetch<SCHEME == GCC_DET ? 1u : 4u> F{&a};
    group_loop<SCHEME, Work>(F, L, S, a.max_ops, deadline, c);
    c.atomics += L.n_atom;
    flush_counters(a.st, c);
}

template <int SCHEME, class Work>
cudaError_t launch_exec(const ExecArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
    auto k = exec_kernel<SCHEME, Work>;
    if (smem > 40 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// Resident blocks per SM of a kernel for a launch shape (0 = cannot launch).
template <class K>
int occupancy_of(K k, int block, size_t smem) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (smem + fa.sharedSizeBytes > (size_t)optin) return 0;   // cannot launch at all
    // raise the dynamic limit whenever static + dynamic passes the 48 KB default
    if (smem + fa.sharedSizeBytes > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();                              // leave no sticky error behind
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int SCHEME, class Work>
int exec_occupancy(int block, size_t smem) {
    return occupancy_of(exec_kernel<SCHEME, Work>, block, smem);
}

}  // namespace gcc
