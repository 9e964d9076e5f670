// exec_kv.cu -- execute a key-value transaction batch under one scheme.
//
// One persistent kernel per (scheme, slot width).  A warp is split into lane
// groups of G lanes; each group takes the next transaction id from a global
// counter (warp-aggregated), stages its op descriptors in shared memory and
// runs attempts until the transaction commits (restart-until-commit, Sec. IV-A
// "Experimental Procedure").  Op j of a transaction is handled by lane j mod G
// of its group, so the group issues up to G independent record accesses at
// once; group-wide decisions (abort, commit) are ballots over the group.
//
// Schemes (Sec. II and Sec. III-E; word layouts in engine.cuh):
//  * NO_WAIT 2PL  -- shared/exclusive lock per record taken before the access,
//    abort as soon as a lock is unavailable, all locks released at commit or
//    abort (Sec. II-A, Sec. III-E.1).  Writes are buffered and applied while
//    the exclusive locks are held.  Commit order: a counter taken while every
//    lock is held (the lock point).
//  * TO           -- per-record RTS/WTS; a read needs ts > WTS, a write needs
//    ts > RTS and ts > WTS, otherwise abort and restart with a new timestamp;
//    a dirty bit locks uncommitted writes (Sec. II-B, Sec. III-E.2).  Commit
//    order: the timestamp.
//  * OCC          -- read phase into a private workspace with version
//    checks, lock the write set without waiting (abort if locked), take a
//    commit timestamp, validate the read set, write and release with the new
//    version (Sec. II-B, Sec. III-E.2 Silo: lock bit + 63-bit timestamp, no
//    epochs, no-wait locking).  Commit order: the timestamp.
//  * DET          -- every op waits until the lower-id accesses to its record
//    that conflict with it are done, then runs; nothing aborts and the outcome
//    is the serial execution in transaction-id order (Sec. II-C GPUTx;
//    Sec. III-E.3 access tables).  Commit order: transaction id.
#include <cstdio>

#include "engine.cuh"

namespace gcc {
namespace {

constexpr uint32_t KIND_SHIFT = 40;
constexpr uint32_t FIELD_SHIFT = 32;

__device__ __forceinline__ uint32_t op_key(uint64_t d) { return (uint32_t)d; }
__device__ __forceinline__ uint32_t op_field(uint64_t d) { return (uint32_t)(d >> FIELD_SHIFT) & 0xffu; }
__device__ __forceinline__ uint32_t op_kind(uint64_t d) { return (uint32_t)(d >> KIND_SHIFT) & 0xffu; }

template <int FB> struct Slot;

template <> struct Slot<8> {
    static __device__ __forceinline__ ulonglong2 load(const uint8_t* p) {
        return make_ulonglong2(ld_relaxed(reinterpret_cast<const uint64_t*>(p)), 0ull);
    }
    static __device__ __forceinline__ void store(uint8_t* p, ulonglong2 v) {
        st_relaxed(reinterpret_cast<uint64_t*>(p), v.x);
    }
    static __device__ __forceinline__ ulonglong2 add(ulonglong2 v, ulonglong2 d) {
        return make_ulonglong2(v.x + d.x, 0ull);
    }
};

template <> struct Slot<16> {
    static __device__ __forceinline__ ulonglong2 load(const uint8_t* p) { return ld_slot16(p); }
    static __device__ __forceinline__ void store(uint8_t* p, ulonglong2 v) { st_slot16(p, v); }
    // lane 0 modulo 2^64; bytes 8-9 as a u16 modulo 2^16; bytes 10-15 kept
    static __device__ __forceinline__ ulonglong2 add(ulonglong2 v, ulonglong2 d) {
        return make_ulonglong2(v.x + d.x, (v.y & ~0xFFFFull) | ((v.y + d.y) & 0xFFFFull));
    }
};

// Per-group view of its shared-memory staging area.
struct Stage {
    uint64_t* desc;
    uint64_t* obs;
    ulonglong2* oldv;
    ulonglong2* newv;
};

struct Lane {
    uint32_t lane, lig, G, gbase;
    unsigned gmask;
};

template <int FB>
__device__ __forceinline__ uint8_t* slot_ptr(const ExecArgs& a, uint32_t key, uint32_t field) {
    return a.table + ((uint64_t)field * a.n_records + key) * FB;
}

__device__ __forceinline__ bool collapse_loser(const ExecArgs& a, uint32_t key) {
    if (a.collapse != 1) return false;
    unsigned am = __activemask();
    unsigned peers = __match_any_sync(am, key);
    return (peers & lanemask_lt()) != 0;
}

__device__ __forceinline__ bool injected_abort(const ExecArgs& a, uint32_t t, uint32_t attempt) {
    if (a.inject_ppm == 0) return false;
    uint64_t h = mix64(a.seed ^ (0x9E3779B97F4A7C15ull * (t + 1)) ^ ((uint64_t)attempt << 40));
    return (uint32_t)(h % 1000000ull) < a.inject_ppm;
}

__device__ __forceinline__ unsigned long long group_ticket(const Lane& L, unsigned long long* ctr) {
    unsigned long long v = 0;
    if (L.lig == 0) v = agg_ticket(ctr);
    return __shfl_sync(L.gmask, v, L.gbase);
}

enum { ABORT = 0, COMMIT = 1, GIVE_UP = 2 };

// ---------------------------------------------------------------------------
// OCC
// ---------------------------------------------------------------------------
template <int FB>
__device__ int occ_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, uint32_t attempt,
                           unsigned long long& order_key) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    // read phase: consistent (version, value) pairs into the workspace
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            uint64_t* m = a.meta + op_key(d);
            const uint8_t* p = slot_ptr<FB>(a, op_key(d), op_field(d));
            for (uint32_t tries = 0;; ++tries) {
                const uint64_t v1 = ld_acquire(m);
                if (!(v1 & OCC_LOCK)) {
                    const ulonglong2 v = Slot<FB>::load(p);
                    __threadfence();
                    if (ld_relaxed(m) == v1) {
                        S.obs[j] = v1;
                        S.oldv[j] = v;
                        if (op_kind(d) == GCC_OP_ADD)
                            S.newv[j] = Slot<FB>::add(v, a.operands[first + j]);
                        break;
                    }
                }
                if (tries >= a.read_retries) { fail = true; break; }
            }
        }
        if (__any_sync(L.gmask, fail)) return ABORT;
    }
    // lock the write set, no waiting; a changed version fails the CAS too
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops && op_kind(S.desc[j]) == GCC_OP_ADD) {
            const uint32_t key = op_key(S.desc[j]);
            bool ok = !collapse_loser(a, key);
            if (ok) ok = cas64(a.meta + key, S.obs[j], S.obs[j] | OCC_LOCK) == S.obs[j];
            if (ok) held |= 1ull << k; else fail = true;
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        __threadfence();
        const unsigned long long ts = group_ticket(L, &a.dbs->occ_clock);
        // validate the read set against the versions observed
        for (uint32_t k = 0; k < kmax; ++k) {
            const uint32_t j = L.lig + k * L.G;
            if (j < nops && op_kind(S.desc[j]) == GCC_OP_READ)
                if (ld_relaxed(a.meta + op_key(S.desc[j])) != S.obs[j]) fail = true;
        }
        if (!__any_sync(L.gmask, fail)) {
            // write phase, then publish the new version and unlock
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) {
                    const uint32_t j = L.lig + k * L.G;
                    Slot<FB>::store(slot_ptr<FB>(a, op_key(S.desc[j]), op_field(S.desc[j])), S.newv[j]);
                }
            __threadfence();
            for (uint32_t k = 0; k < kmax; ++k)
                if (held >> k & 1) st_relaxed(a.meta + op_key(S.desc[L.lig + k * L.G]), ts + 1);
            order_key = ts;
            return COMMIT;
        }
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            st_release(a.meta + op_key(S.desc[j]), S.obs[j]);
        }
    return ABORT;
}

// ---------------------------------------------------------------------------
// NO_WAIT 2PL
// ---------------------------------------------------------------------------
template <int FB>
__device__ int tpl_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, uint32_t attempt,
                           unsigned long long& order_key) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            uint64_t* m = a.meta + op_key(d);
            if (op_kind(d) == GCC_OP_READ) {
                for (uint32_t tries = 0;; ++tries) {
                    const uint64_t w = ld_relaxed(m);
                    if (w & TPL_X) { fail = true; break; }
                    if (cas64(m, w, w + TPL_S_ONE) == w) { held |= 1ull << k; break; }
                    if (tries >= a.read_retries) { fail = true; break; }
                }
            } else {
                bool ok = !collapse_loser(a, op_key(d));
                if (ok) ok = cas64(m, 0ull, TPL_X | (uint64_t)(t + 1)) == 0ull;
                if (ok) held |= 1ull << k; else fail = true;
            }
            if (!fail) {
                __threadfence();
                const ulonglong2 v = Slot<FB>::load(slot_ptr<FB>(a, op_key(d), op_field(d)));
                S.oldv[j] = v;
                if (op_kind(d) == GCC_OP_ADD) S.newv[j] = Slot<FB>::add(v, a.operands[first + j]);
            }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        // lock point: every lock is held
        const unsigned long long ts = group_ticket(L, &a.st->ticket);
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                if (op_kind(S.desc[j]) == GCC_OP_ADD)
                    Slot<FB>::store(slot_ptr<FB>(a, op_key(S.desc[j]), op_field(S.desc[j])), S.newv[j]);
            }
        __threadfence();
        order_key = ts;
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            uint64_t* m = a.meta + op_key(S.desc[j]);
            if (op_kind(S.desc[j]) == GCC_OP_READ) add64(m, (uint64_t)0 - TPL_S_ONE);
            else st_release(m, 0ull);
        }
    return fail ? ABORT : COMMIT;
}

// ---------------------------------------------------------------------------
// basic TO
// ---------------------------------------------------------------------------
template <int FB>
__device__ int to_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                          uint64_t first, uint32_t nops, uint32_t attempt,
                          unsigned long long& order_key) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    const unsigned long long ts = group_ticket(L, &a.st->ticket) + 1;
    if (ts > TO_TS_MASK) {
        if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_TS_OVERFLOW);
        return GIVE_UP;
    }
    bool fail = false;
    uint64_t held = 0;
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            uint64_t* m = a.meta + op_key(d);
            const uint8_t* p = slot_ptr<FB>(a, op_key(d), op_field(d));
            if (op_kind(d) == GCC_OP_READ) {
                for (uint32_t tries = 0;; ++tries) {
                    const uint64_t w = ld_acquire(m);
                    const uint64_t wts = w & TO_TS_MASK, rts = (w >> TO_RTS_SHIFT) & TO_TS_MASK;
                    if ((w & TO_DIRTY) || ts < wts) { fail = true; break; }
                    const ulonglong2 v = Slot<FB>::load(p);
                    __threadfence();
                    bool ok;
                    if (rts >= ts) {
                        ok = ld_relaxed(m) == w;
                    } else {
                        const uint64_t nw = (w & ~(TO_TS_MASK << TO_RTS_SHIFT)) | (ts << TO_RTS_SHIFT);
                        ok = cas64(m, w, nw) == w;
                    }
                    if (ok) { S.oldv[j] = v; break; }
                    if (tries >= a.read_retries) { fail = true; break; }
                }
            } else {
                bool ok = !collapse_loser(a, op_key(d));
                for (uint32_t tries = 0; ok; ++tries) {
                    const uint64_t w = ld_relaxed(m);
                    const uint64_t wts = w & TO_TS_MASK, rts = (w >> TO_RTS_SHIFT) & TO_TS_MASK;
                    if ((w & TO_DIRTY) || ts < rts || ts < wts) { ok = false; break; }
                    const uint64_t nw = TO_DIRTY | (rts << TO_RTS_SHIFT) | ts;
                    if (cas64(m, w, nw) == w) { S.obs[j] = w; break; }
                    if (tries >= a.read_retries) { ok = false; break; }
                }
                if (ok) {
                    held |= 1ull << k;
                    __threadfence();
                    const ulonglong2 v = Slot<FB>::load(p);
                    S.oldv[j] = v;
                    S.newv[j] = Slot<FB>::add(v, a.operands[first + j]);
                } else {
                    fail = true;
                }
            }
        }
        if (__any_sync(L.gmask, fail)) break;
    }
    fail = __any_sync(L.gmask, fail) || injected_abort(a, t, attempt);
    if (!fail) {
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                Slot<FB>::store(slot_ptr<FB>(a, op_key(S.desc[j]), op_field(S.desc[j])), S.newv[j]);
            }
        __threadfence();
        for (uint32_t k = 0; k < kmax; ++k)
            if (held >> k & 1) {
                const uint32_t j = L.lig + k * L.G;
                st_relaxed(a.meta + op_key(S.desc[j]),
                           (S.obs[j] & (TO_TS_MASK << TO_RTS_SHIFT)) | ts);
            }
        order_key = ts;
        return COMMIT;
    }
    for (uint32_t k = 0; k < kmax; ++k)
        if (held >> k & 1) {
            const uint32_t j = L.lig + k * L.G;
            st_release(a.meta + op_key(S.desc[j]), S.obs[j]);
        }
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

// An invalid transaction never runs, but its accesses are in the batch's
// access table: advance its records' counters in order so that later
// transactions on those records are not held up.
__device__ void det_skip(const ExecArgs& a, const Lane& L, uint64_t first, uint32_t nops) {
    if (first + nops > a.n_ops) return;
    for (uint32_t j = L.lig; j < nops; j += L.G) {
        const uint64_t d = a.ops[first + j];
        const uint32_t rec = cc_record(d, GCC_SCHEMA_KV, 0, 0xffffffffu);
        if (rec >= a.n_meta) continue;
        const bool w = kind_writes(op_kind(d));
        if (det_wait(a, a.meta + rec, w, a.need[first + j]))
            add64(a.meta + rec, w ? DET_WRITE_DONE : DET_READ_DONE);
    }
}

template <int FB>
__device__ int det_attempt(const ExecArgs& a, const Lane& L, const Stage& S, uint32_t t,
                           uint64_t first, uint32_t nops, unsigned long long& order_key) {
    const uint32_t kmax = (nops + L.G - 1) / L.G;
    bool fail = false;
    for (uint32_t k = 0; k < kmax && !fail; ++k) {
        const uint32_t j = L.lig + k * L.G;
        if (j < nops) {
            const uint64_t d = S.desc[j];
            uint64_t* m = a.meta + op_key(d);
            const bool w = op_kind(d) == GCC_OP_ADD;
            if (!det_wait(a, m, w, a.need[first + j])) { fail = true; break; }
            uint8_t* p = slot_ptr<FB>(a, op_key(d), op_field(d));
            const ulonglong2 v = Slot<FB>::load(p);
            S.oldv[j] = v;
            if (w) Slot<FB>::store(p, Slot<FB>::add(v, a.operands[first + j]));
            __threadfence();
            add64(m, w ? DET_WRITE_DONE : DET_READ_DONE);
        }
    }
    if (__any_sync(L.gmask, fail)) return GIVE_UP;
    order_key = t;
    return COMMIT;
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int SCHEME, int FB>
__global__ void __launch_bounds__(1024) kv_exec_kernel(const ExecArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    Lane L;
    L.G = a.lanes;
    L.lane = threadIdx.x & 31;
    L.lig = L.lane & (L.G - 1);
    L.gbase = L.lane & ~(L.G - 1);
    L.gmask = (L.G == 32) ? 0xffffffffu : (((1u << L.G) - 1u) << L.gbase);
    const uint32_t slots = blockDim.x / L.G;
    const uint32_t slot = threadIdx.x / L.G;
    const uint32_t M = a.max_ops;
    Stage S;
    uint64_t* w64 = reinterpret_cast<uint64_t*>(smem);
    S.desc = w64 + (size_t)slot * M;
    S.obs = w64 + (size_t)slots * M + (size_t)slot * M;
    ulonglong2* w128 = reinterpret_cast<ulonglong2*>(w64 + 2 * (size_t)slots * M);
    S.oldv = w128 + (size_t)slot * M;
    S.newv = w128 + (size_t)slots * M + (size_t)slot * M;

    const uint64_t deadline = globaltimer() + a.deadline_ns;
    unsigned commits = 0, aborts = 0, timeouts = 0, invalid = 0, max_att = 0;

    for (;;) {
        unsigned long long tt = 0;
        if (L.lig == 0) tt = agg_ticket(&a.st->fetch);
        tt = __shfl_sync(L.gmask, tt, L.gbase);
        if (tt >= a.n_txns) break;
        const uint32_t t = (uint32_t)tt;
        const gcc_txn tx = a.txns[t];
        const uint32_t nops = tx.n_ops;
        const uint64_t first = tx.first_op;
        bool bad = nops > M || tx.type != GCC_TXN_KV || first + nops > a.n_ops;
        if (!bad) {
            for (uint32_t j = L.lig; j < nops; j += L.G) {
                const uint64_t d = a.ops[first + j];
                S.desc[j] = d;
                if (op_key(d) >= a.n_records || op_field(d) >= a.n_fields ||
                    (op_kind(d) != GCC_OP_READ && op_kind(d) != GCC_OP_ADD))
                    bad = true;
            }
        }
        __syncwarp(L.gmask);
        if (!__any_sync(L.gmask, bad)) {
            for (uint32_t j = L.lig; j < nops; j += L.G)
                for (uint32_t i = 0; i < j; ++i)
                    if (op_key(S.desc[i]) == op_key(S.desc[j])) bad = true;
        }
        if (__any_sync(L.gmask, bad)) {
            if constexpr (SCHEME == GCC_DET) det_skip(a, L, first, nops);
            if (L.lig == 0) {
                a.results[t] = gcc_txn_result{GCC_TXN_INVALID, 0u, ~0ull};
                atomicOr(&a.st->error, GCC_DEVERR_INVALID);
                ++invalid;
            }
            __syncwarp(L.gmask);
            continue;
        }

        uint32_t attempts = 0;
        int outcome = ABORT;
        unsigned long long order_key = 0;
        for (;;) {
            ++attempts;
            if constexpr (SCHEME == GCC_OCC)
                outcome = occ_attempt<FB>(a, L, S, t, first, nops, attempts, order_key);
            else if constexpr (SCHEME == GCC_NO_WAIT_2PL)
                outcome = tpl_attempt<FB>(a, L, S, t, first, nops, attempts, order_key);
            else if constexpr (SCHEME == GCC_TO)
                outcome = to_attempt<FB>(a, L, S, t, first, nops, attempts, order_key);
            else
                outcome = det_attempt<FB>(a, L, S, t, first, nops, order_key);
            if (outcome != ABORT) break;
            if (L.lig == 0) ++aborts;
            if (attempts >= a.max_attempts) {
                if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_ATTEMPTS);
                outcome = GIVE_UP;
                break;
            }
            if (globaltimer() > deadline) {
                if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_DEADLINE);
                outcome = GIVE_UP;
                break;
            }
            if (a.backoff_base_ns) {
                const uint32_t sh = attempts - 1 < 16 ? attempts - 1 : 16;
                uint64_t d = (uint64_t)a.backoff_base_ns << sh;
                if (d > a.backoff_cap_ns) d = a.backoff_cap_ns;
                d = d / 2 + mix64(a.seed ^ ((uint64_t)t << 20) ^ attempts) % (d / 2 + 1);
                while (d > 0) {
                    const uint32_t s = d > 100000 ? 100000u : (uint32_t)d;
                    __nanosleep(s);
                    d -= s;
                }
            }
        }
        if (outcome == COMMIT) {
            for (uint32_t j = L.lig; j < nops; j += L.G) a.reads[first + j] = S.oldv[j];
            if (L.lig == 0) {
                // 2PL tickets are dense already; OCC/TO keys are densified later
                const bool dense = SCHEME == GCC_NO_WAIT_2PL || SCHEME == GCC_DET;
                a.results[t] = gcc_txn_result{GCC_TXN_COMMITTED, attempts,
                                              dense ? (uint64_t)order_key : ~0ull};
                if (!dense) a.order_key[t] = order_key;
                ++commits;
            }
        } else if (L.lig == 0) {
            a.results[t] = gcc_txn_result{GCC_TXN_TIMEOUT, attempts, ~0ull};
            if (!(SCHEME == GCC_NO_WAIT_2PL || SCHEME == GCC_DET)) a.order_key[t] = ~0ull;
            ++timeouts;
        }
        if (L.lig == 0 && attempts > max_att) max_att = attempts;
        __syncwarp(L.gmask);
    }
    // one atomic per warp and counter
    commits = __reduce_add_sync(0xffffffffu, commits);
    aborts = __reduce_add_sync(0xffffffffu, aborts);
    timeouts = __reduce_add_sync(0xffffffffu, timeouts);
    invalid = __reduce_add_sync(0xffffffffu, invalid);
    max_att = __reduce_max_sync(0xffffffffu, max_att);
    if ((threadIdx.x & 31) == 0) {
        if (commits) atomicAdd(&a.st->committed, (unsigned long long)commits);
        if (aborts) atomicAdd(&a.st->aborts, (unsigned long long)aborts);
        if (timeouts) atomicAdd(&a.st->timeouts, (unsigned long long)timeouts);
        if (invalid) atomicAdd(&a.st->invalid, (unsigned long long)invalid);
        if (max_att) atomicMax(&a.st->max_attempts, (unsigned long long)max_att);
    }
}

template <int SCHEME, int FB>
cudaError_t launch_one(const ExecArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
    auto k = kv_exec_kernel<SCHEME, FB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SCHEME, int FB>
int occupancy_one(int block, size_t smem) {
    auto k = kv_exec_kernel<SCHEME, FB>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess) return 0;
    return n;
}

}  // namespace

cudaError_t launch_kv_exec(gcc_scheme scheme, uint32_t fb, const ExecArgs& a, int grid,
                           int block, size_t smem, cudaStream_t s) {
#define GCC_KV_CASE(SC)                                                      \
    case SC:                                                                 \
        return fb == 16 ? launch_one<SC, 16>(a, grid, block, smem, s)        \
                        : launch_one<SC, 8>(a, grid, block, smem, s);
    switch (scheme) {
        GCC_KV_CASE(GCC_NO_WAIT_2PL)
        GCC_KV_CASE(GCC_TO)
        GCC_KV_CASE(GCC_OCC)
        GCC_KV_CASE(GCC_DET)
    }
#undef GCC_KV_CASE
    return cudaErrorInvalidValue;
}

int kv_exec_occupancy(gcc_scheme scheme, uint32_t fb, int block, size_t smem) {
#define GCC_KV_OCC(SC) \
    case SC: return fb == 16 ? occupancy_one<SC, 16>(block, smem) : occupancy_one<SC, 8>(block, smem);
    switch (scheme) {
        GCC_KV_OCC(GCC_NO_WAIT_2PL)
        GCC_KV_OCC(GCC_TO)
        GCC_KV_OCC(GCC_OCC)
        GCC_KV_OCC(GCC_DET)
    }
#undef GCC_KV_OCC
    return 0;
}

}  // namespace gcc
