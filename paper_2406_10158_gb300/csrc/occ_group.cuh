// occ_group.cuh -- OCC with group commit on key-value batches.
//
// The chain of commits on a contended record is serial: every committed
// write of it is one tenure of its lock, and on GB300 one tenure (lock CAS,
// acquire-release commit timestamp, validation, write, release publish) is
// about 3.7 us of dependent round trips.  Group commit puts several
// transactions that write the same contended record into one unit, and a
// lane group runs the unit as one OCC attempt (Sec. II-B, Sec. III-E.2 Silo,
// applied to the unit):
//   1. read phase over every op of the pending members: versions (relaxed,
//      all in flight), one acquire fence, then the values;
//   2. one no-wait lock CAS per distinct written record of the unit, from
//      the version its lowest op observed; a member whose written record could
//      not be locked drops out of this attempt;
//   3. one acquire-release atomic takes consecutive commit timestamps for the
//      remaining members, in member order;
//   4. each member validates its reads of records the unit does not hold;
//      one that fails drops out (its timestamp stays unused);
//   5. every held record is evaluated in timestamp order over the members
//      that commit: a member's read of it returns the value after the earlier
//      members' writes, its write applies on top; the record is written once
//      and published once with the last writer's timestamp + 1.
// The unit holds every record it writes from step 2 to step 5 and takes its
// timestamps while holding them, so it is serializable as one transaction
// whose members follow each other in timestamp order: each member's result is
// the serial execution in commit order.  Members that dropped out retry in
// the unit's next attempt, after the randomized backoff of the plain kernel
// (and, once the unit has failed queue_after times, a turn in the retry
// queue of the record it failed on); a member is never waited for.
//
// Units are formed before the launch (occ_group.cu): each transaction is
// keyed by its written record with the most writes in the batch, if no other
// record it touches is contended too; the transactions of one key, in id
// order, are cut into units of up to U.  A unit is run by whichever group
// fetches its lowest id; its other members' ids are skipped when fetched.
#pragma once

#include "exec_common.cuh"

namespace gcc {

constexpr uint32_t UNIT_NONE = 0x7fffffffu;      // no next member
constexpr uint32_t UNIT_FOLLOWER = 0x80000000u;  // runs with a lower id's unit
constexpr uint32_t HEMPTY = 0xffffffffu;

// Shared-memory layout of one lane group's unit (U members of up to M ops).
struct UnitLayout {
    uint32_t U, M, UOPS, H;
    __host__ __device__ static uint32_t hash_size(uint32_t uops) {
        uint32_t h = 32;
        while (h < 2 * uops) h <<= 1;
        return h;
    }
    __host__ __device__ UnitLayout(uint32_t u, uint32_t m) : U(u), M(m), UOPS(u * m),
                                                             H(hash_size(u * m)) {}
    // byte offsets inside the group's slot, largest alignment first
    __host__ __device__ size_t off_oldv() const { return 0; }
    __host__ __device__ size_t off_desc() const { return off_oldv() + (size_t)UOPS * 16; }
    __host__ __device__ size_t off_obs() const { return off_desc() + (size_t)UOPS * 8; }
    __host__ __device__ size_t off_mfirst() const { return off_obs() + (size_t)UOPS * 8; }
    __host__ __device__ size_t off_hkey() const { return off_mfirst() + (size_t)U * 8; }
    __host__ __device__ size_t off_hrep() const { return off_hkey() + (size_t)H * 4; }
    __host__ __device__ size_t off_hst() const { return off_hrep() + (size_t)H * 4; }
    __host__ __device__ size_t off_mt() const { return off_hst() + (size_t)H * 4; }
    __host__ __device__ size_t off_moff() const { return off_mt() + (size_t)U * 4; }
    __host__ __device__ size_t off_matt() const { return off_moff() + (size_t)(U + 1) * 4; }
    __host__ __device__ size_t off_flags() const { return off_matt() + (size_t)U * 4; }
    __host__ __device__ size_t off_hent() const { return off_flags() + 4 * 4; }
    __host__ __device__ size_t off_mof() const { return off_hent() + (size_t)UOPS * 2; }
    __host__ __device__ size_t off_hopm() const { return off_mof() + (size_t)UOPS; }
    __host__ __device__ size_t bytes() const {
        return (off_hopm() + (size_t)H * U + 15) & ~(size_t)15;
    }
};

struct UnitStage {
    ulonglong2* oldv;   // [UOPS] value read (then the value the member's op returns)
    uint64_t* desc;     // [UOPS] op descriptors, members one after another
    uint64_t* obs;      // [UOPS] version observed (OCC_LOCK set: the read failed)
    uint64_t* mfirst;   // [U] first op index of each member in the batch
    uint32_t* hkey;     // [H] record of each entry (HEMPTY: free)
    uint32_t* hrep;     // [H] lowest pending op on the record: it locks the record
    uint32_t* hst;      // [H] 1: a pending op writes it; 2: held by the unit; 4: lock failed
    uint32_t* mt;       // [U] transaction ids
    uint32_t* moff;     // [U + 1] op offsets of the members
    uint32_t* matt;     // [U] attempts of each member
    uint32_t* flags;    // [0]: members dropped out of the current attempt;
                        // [2]: lowest op that made one drop out (HEMPTY: none)
    uint16_t* hent;     // [UOPS] entry of each op's record
    uint8_t* mof;       // [UOPS] member of each op
    uint8_t* hopm;      // [H * U] op of member m on the entry's record (0xff: none)
    UnitLayout lay;
    __device__ UnitStage() : lay(1, 1) {}
};

__device__ __forceinline__ void setup_unit_stage(const ExecArgs& a, const Lane& L, UnitStage& S) {
    extern __shared__ __align__(16) unsigned char smem[];
    S.lay = UnitLayout(a.group_u, a.max_ops);
    const uint32_t slot = threadIdx.x / L.G;
    unsigned char* b = smem + (size_t)slot * S.lay.bytes();
    S.oldv = reinterpret_cast<ulonglong2*>(b + S.lay.off_oldv());
    S.desc = reinterpret_cast<uint64_t*>(b + S.lay.off_desc());
    S.obs = reinterpret_cast<uint64_t*>(b + S.lay.off_obs());
    S.mfirst = reinterpret_cast<uint64_t*>(b + S.lay.off_mfirst());
    S.hkey = reinterpret_cast<uint32_t*>(b + S.lay.off_hkey());
    S.hrep = reinterpret_cast<uint32_t*>(b + S.lay.off_hrep());
    S.hst = reinterpret_cast<uint32_t*>(b + S.lay.off_hst());
    S.mt = reinterpret_cast<uint32_t*>(b + S.lay.off_mt());
    S.moff = reinterpret_cast<uint32_t*>(b + S.lay.off_moff());
    S.matt = reinterpret_cast<uint32_t*>(b + S.lay.off_matt());
    S.flags = reinterpret_cast<uint32_t*>(b + S.lay.off_flags());
    S.hent = reinterpret_cast<uint16_t*>(b + S.lay.off_hent());
    S.mof = reinterpret_cast<uint8_t*>(b + S.lay.off_mof());
    S.hopm = reinterpret_cast<uint8_t*>(b + S.lay.off_hopm());
}

__device__ __forceinline__ unsigned long long ticket_acq_rel_n(unsigned long long* ctr, uint32_t n) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                 : "=l"(old) : "l"(ctr), "l"((unsigned long long)n) : "memory");
    return old;
}

// Entry table of the unit's records, built once per unit (members fixed).
template <class Work>
__device__ void unit_build_table(const ExecArgs& a, const Lane& L, const UnitStage& S, uint32_t nu) {
    const UnitLayout& y = S.lay;
    for (uint32_t e = L.lig; e < y.H; e += L.G) {
        S.hkey[e] = HEMPTY;
        for (uint32_t m = 0; m < y.U; ++m) S.hopm[e * y.U + m] = 0xff;
    }
    __syncwarp(L.gmask);
    for (uint32_t j = L.lig; j < nu; j += L.G) {
        const uint32_t r = Work::rec(a, S.desc[j]);
        uint32_t e = ((r * 2654435761u) >> 16) & (y.H - 1);
        for (uint32_t probe = 0; probe < y.H; ++probe) {
            const uint32_t old = atomicCAS(&S.hkey[e], HEMPTY, r);
            if (old == HEMPTY || old == r) break;
            e = (e + 1) & (y.H - 1);
        }
        S.hent[j] = (uint16_t)e;
        S.hopm[e * y.U + S.mof[j]] = (uint8_t)j;
    }
    __syncwarp(L.gmask);
}

// Per-op loops below take a lane's ops four at a time, with the four memory
// operations issued before any result is used, so that they are in flight
// together.
constexpr uint32_t UQ = 4;

// One attempt of the unit's pending members.  Returns the members that
// committed; `taken` are the members that took a timestamp (member m's is
// tbase + the number of members in `taken` below m).
template <class Work>
__device__ uint32_t unit_attempt(const ExecArgs& a, const Lane& L, const UnitStage& S,
                                 uint32_t nmem, uint32_t nu, uint32_t pend,
                                 unsigned long long& tbase, uint32_t& taken) {
    const UnitLayout& y = S.lay;
    const uint32_t kmax = (nu + L.G - 1) / L.G;
    auto op_at = [&](uint32_t k) -> uint32_t { return L.lig + k * L.G; };
    auto live = [&](uint32_t j) -> bool { return j < nu && (pend >> S.mof[j] & 1); };

    // 0. per-attempt entry state over the pending members' ops
    for (uint32_t e = L.lig; e < y.H; e += L.G) { S.hst[e] = 0; S.hrep[e] = HEMPTY; }
    if (L.lig == 0) { S.flags[0] = 0; S.flags[2] = HEMPTY; }
    __syncwarp(L.gmask);
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = op_at(k);
        if (live(j)) {
            const uint32_t e = S.hent[j];
            atomicMin(&S.hrep[e], j);
            if (Work::writes(S.desc[j])) atomicOr(&S.hst[e], 1u);
        }
    }
    // 1. read phase: versions in flight together, one fence, then the values
    for (uint32_t k0 = 0; k0 < kmax; k0 += UQ) {
        uint64_t v[UQ];
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            v[q] = (k0 + q < kmax && live(j)) ? ld_relaxed(a.meta + Work::rec(a, S.desc[j])) : 0ull;
        }
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            if (k0 + q < kmax && live(j)) S.obs[j] = v[q];
        }
    }
    fence_acq_rel();
    for (uint32_t k0 = 0; k0 < kmax; k0 += UQ) {
        ulonglong2 v[UQ];
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            v[q] = (k0 + q < kmax && live(j) && !(S.obs[j] & OCC_LOCK)) ? Work::load(a, S.desc[j])
                                                                        : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            if (k0 + q < kmax && live(j)) S.oldv[j] = v[q];
        }
    }
    // a record seen locked: re-read a few times, then the member drops out
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = op_at(k);
        if (live(j) && (S.obs[j] & OCC_LOCK)) {
            const uint64_t d = S.desc[j];
            uint64_t v1 = S.obs[j];
            for (uint32_t tries = 0; (v1 & OCC_LOCK) && tries < a.read_retries; ++tries) {
                __nanosleep(32);
                v1 = ld_acquire(a.meta + Work::rec(a, d));
            }
            S.obs[j] = v1;
            if (!(v1 & OCC_LOCK)) {
                S.oldv[j] = Work::load(a, d);
            } else {
                atomicOr(&S.flags[0], 1u << S.mof[j]);
                atomicMin(&S.flags[2], j);
            }
        }
    }
    __syncwarp(L.gmask);
    // 2. one lock CAS per written record, by the lane of its lowest pending op
    for (uint32_t k0 = 0; k0 < kmax; k0 += UQ) {
        uint64_t got[UQ];
        bool mine[UQ];
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            mine[q] = k0 + q < kmax && live(j) && S.hrep[S.hent[j]] == j && (S.hst[S.hent[j]] & 1u);
            got[q] = 0;
            if (mine[q] && !(S.obs[j] & OCC_LOCK)) {
                ++L.n_atom;
                got[q] = cas64(a.meta + Work::rec(a, S.desc[j]), S.obs[j], S.obs[j] | OCC_LOCK);
            }
        }
#pragma unroll
        for (uint32_t q = 0; q < UQ; ++q) {
            const uint32_t j = op_at(k0 + q);
            if (mine[q]) {
                const bool ok = !(S.obs[j] & OCC_LOCK) && got[q] == S.obs[j];
                atomicOr(&S.hst[S.hent[j]], ok ? 2u : 4u);
            }
        }
    }
    __syncwarp(L.gmask);
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = op_at(k);
        if (live(j) && Work::writes(S.desc[j]) && !(S.hst[S.hent[j]] & 2u)) {
            atomicOr(&S.flags[0], 1u << S.mof[j]);
            atomicMin(&S.flags[2], j);
        }
    }
    __syncwarp(L.gmask);
    for (uint32_t m = L.lig; m < nmem; m += L.G)
        if ((pend >> m & 1) && injected_abort(a, S.mt[m], S.matt[m])) atomicOr(&S.flags[0], 1u << m);
    __syncwarp(L.gmask);
    uint32_t alive = pend & ~S.flags[0];
    __syncwarp(L.gmask);
    // 3. consecutive timestamps for the members still in, in member order;
    // the acquire-release atomic orders the unit's locks before it and the
    // validation after it (the warp barrier brings the other lanes' locks)
    tbase = 0;
    taken = alive;
    if (alive) {
        unsigned long long b = 0;
        if (L.lig == 0) { b = ticket_acq_rel_n(&a.dbs->occ_clock, __popc(alive)); ++L.n_atom; }
        tbase = __shfl_sync(L.gmask, b, L.gbase);
        __syncwarp(L.gmask);
        // 4. validate reads of records the unit does not hold
        for (uint32_t k0 = 0; k0 < kmax; k0 += UQ) {
            uint64_t v[UQ];
            bool chk[UQ];
#pragma unroll
            for (uint32_t q = 0; q < UQ; ++q) {
                const uint32_t j = op_at(k0 + q);
                chk[q] = k0 + q < kmax && j < nu && (alive >> S.mof[j] & 1) &&
                         !(S.hst[S.hent[j]] & 2u);
                v[q] = chk[q] ? ld_relaxed(a.meta + Work::rec(a, S.desc[j])) : 0ull;
            }
#pragma unroll
            for (uint32_t q = 0; q < UQ; ++q) {
                const uint32_t j = op_at(k0 + q);
                if (chk[q] && v[q] != S.obs[j]) {
                    atomicOr(&S.flags[0], 1u << S.mof[j]);
                    atomicMin(&S.flags[2], j);
                }
            }
        }
        __syncwarp(L.gmask);
        alive = pend & ~S.flags[0];
        __syncwarp(L.gmask);
    }
    // 5. every held record in timestamp order over the committing members,
    // written and published once (released unchanged when none of them
    // writes it)
    for (uint32_t k = 0; k < kmax; ++k) {
        const uint32_t j = op_at(k);
        if (!live(j)) continue;
        const uint32_t e = S.hent[j];
        if (S.hrep[e] != j || !(S.hst[e] & 2u)) continue;
        const uint64_t v0 = S.obs[j];
        uint64_t* mw = a.meta + Work::rec(a, S.desc[j]);
        // at most one op per member on a record: at most U (<= 8) fields
        uint32_t nf = 0;
        uint32_t fld[8];
        ulonglong2 cur[8];
        uint32_t lastw[8];
        bool any_w = false;
        unsigned long long last_ts = 0;
        for (uint32_t m = 0; m < nmem; ++m) {
            const uint32_t o = S.hopm[e * y.U + m];
            if (o == 0xff || !(alive >> m & 1)) continue;
            const uint64_t d = S.desc[o];
            const uint32_t f = op_field(d);
            uint32_t i = 0;
            while (i < nf && fld[i] != f) ++i;
            if (i == nf) {
                // the field's value at the lock: an op that saw the locked
                // version read it; otherwise read it now (the record is held)
                fld[nf] = f;
                cur[nf] = (S.obs[o] == v0) ? S.oldv[o] : Work::load(a, d);
                lastw[nf] = 0xffffffffu;
                ++nf;
            }
            S.oldv[o] = cur[i];
            if (Work::writes(d)) {
                const uint64_t gi = S.mfirst[m] + (o - S.moff[m]);
                cur[i] = Work::compute(a, d, cur[i], a.operands[gi]);
                lastw[i] = o;
                any_w = true;
                last_ts = tbase + __popc(taken & ((1u << m) - 1u));
            }
        }
        for (uint32_t i = 0; i < nf; ++i)
            if (lastw[i] != 0xffffffffu) Work::store(a, S.desc[lastw[i]], cur[i], 0);
        st_release(mw, any_w ? last_ts + 1 : v0);
    }
    __syncwarp(L.gmask);
    return alive;
}

// The execution loop of one lane group under group commit: take a unit,
// stage and check its members, attempt it until every member committed or
// gave up.
template <class Fetch, class Work>
__device__ void unit_loop(Fetch& F, const Lane& L, const UnitStage& S, uint64_t deadline,
                          Counters& c) {
    const UnitLayout& y = S.lay;
    bool finished = false, has = false, served = false;
    uint32_t nmem = 0, nu = 0, pend = 0, uatt = 0;
    uint64_t wake = 0;
    uint32_t qi = NO_Q, qt = 0;   // retry queue and ticket while queued
    uint32_t pq = NO_Q;           // queue to join once the backoff is over
    const ExecArgs* A = nullptr;
    for (;;) {
        // 1. a group without a unit takes the next id; a follower's id is
        // skipped (its unit runs where its lowest id was fetched)
        if (!has && !finished) {
            uint32_t t = 0;
            if (!F.next(L, t, A)) {
                finished = true;
            } else {
                const ExecArgs& a = *A;
                uint32_t link = a.unit_link[t];
                if (!(link & UNIT_FOLLOWER)) {
                    nmem = 0;
                    nu = 0;
                    uint32_t cur = t;
                    for (;;) {
                        const gcc_txn tx = a.txns[cur];
                        const uint32_t nops = tx.n_ops;
                        const uint64_t first = tx.first_op;
                        bool bad = nops > y.M || !Work::valid_txn(a, tx) || first + nops > a.n_ops;
                        if (!bad) {
                            for (uint32_t j = L.lig; j < nops; j += L.G) {
                                const uint64_t d = a.ops[first + j];
                                S.desc[nu + j] = d;
                                S.mof[nu + j] = (uint8_t)nmem;
                                if (!Work::valid_op(a, d)) bad = true;
                            }
                        }
                        __syncwarp(L.gmask);
                        if (!__any_sync(L.gmask, bad)) {
                            for (uint32_t j = L.lig; j < nops; j += L.G) {
                                const uint32_t rj = Work::rec(a, S.desc[nu + j]);
                                for (uint32_t i = 0; i < j; ++i)
                                    if (Work::rec(a, S.desc[nu + i]) == rj) bad = true;
                            }
                        }
                        if (__any_sync(L.gmask, bad)) {
                            if (L.lig == 0) {
                                a.results[cur] = gcc_txn_result{GCC_TXN_INVALID, 0u, ~0ull};
                                a.order_key[cur] = ~0ull;
                                atomicOr(&a.st->error, GCC_DEVERR_INVALID);
                                ++c.invalid;
                            }
                        } else {
                            if (L.lig == 0) {
                                S.mt[nmem] = cur;
                                S.mfirst[nmem] = first;
                                S.moff[nmem] = nu;
                                S.matt[nmem] = 0;
                            }
                            ++nmem;
                            nu += nops;
                        }
                        __syncwarp(L.gmask);
                        const uint32_t nx = link & UNIT_NONE;
                        if (nx == UNIT_NONE || nx >= a.n_txns || nmem == y.U) break;
                        cur = nx;
                        link = a.unit_link[cur];
                    }
                    if (L.lig == 0) S.moff[nmem] = nu;
                    __syncwarp(L.gmask);
                    if (nmem) {
                        unit_build_table<Work>(a, L, S, nu);
                        has = true;
                        pend = (nmem == 32) ? 0xffffffffu : ((1u << nmem) - 1u);
                        uatt = 0;
                        wake = 0;
                        qi = pq = NO_Q;
                        served = false;
                    }
                }
            }
        }
        if (__all_sync(0xffffffffu, finished && !has)) break;

        // 2. one attempt per group holding a unit that is neither backing off
        // nor waiting for its turn in a retry queue (the queues of the plain
        // execute kernel: a unit that keeps failing takes a ticket in the
        // queue of the record it failed on)
        const uint64_t now = __shfl_sync(0xffffffffu, globaltimer(), L.gbase);
        bool go = false, expired = false;
        if (has && now < wake) {
        } else if (has && (pq != NO_Q || (qi != NO_Q && !served))) {
            const ExecArgs& a = *A;
            uint64_t w = 0;
            if (pq != NO_Q) {
                qi = pq;
                pq = NO_Q;
                if (L.lig == 0) { w = add64(a.rq + qi, 1ull << 32); ++L.n_atom; }
                w = __shfl_sync(L.gmask, w, L.gbase);
                qt = (uint32_t)(w >> 32);
            } else {
                if (L.lig == 0) w = ld_relaxed(a.rq + qi);
                w = __shfl_sync(L.gmask, w, L.gbase);
            }
            const int32_t ahead = (int32_t)(qt - (uint32_t)w);
            if (ahead < (int32_t)a.queue_width) {
                served = go = true;
            } else if (now > deadline) {
                expired = true;
                qi = NO_Q;
            } else {
                wake = now + queue_wait_ns(a, (uint32_t)(ahead - (int32_t)a.queue_width + 1));
            }
        } else if (has) {
            go = true;
        }
        if (expired) {
            const ExecArgs& a = *A;
            for (uint32_t m = L.lig; m < nmem; m += L.G) {
                if (!(pend >> m & 1)) continue;
                a.results[S.mt[m]] = gcc_txn_result{GCC_TXN_TIMEOUT, S.matt[m], ~0ull};
                a.order_key[S.mt[m]] = ~0ull;
                ++c.timeouts;
                if (S.matt[m] > c.max_att) c.max_att = S.matt[m];
            }
            if (L.lig == 0) atomicOr(&a.st->error, GCC_DEVERR_DEADLINE);
            pend = 0;
            has = false;
            __syncwarp(L.gmask);
        }
        if (go) {
            const ExecArgs& a = *A;
            ++uatt;
            for (uint32_t m = L.lig; m < nmem; m += L.G)
                if (pend >> m & 1) ++S.matt[m];
            __syncwarp(L.gmask);
            unsigned long long tbase = 0;
            uint32_t taken = 0;
            const uint32_t won = unit_attempt<Work>(a, L, S, nmem, nu, pend, tbase, taken);
            const uint32_t fop = S.flags[2];
            const uint32_t crec = fop != HEMPTY ? Work::rec(a, S.desc[fop]) : NO_CC;
            if (served) {                      // pass the queue's turn on
                if (L.lig == 0) { add64(a.rq + qi, 1ull); ++L.n_atom; }
                served = false;
                qi = NO_Q;
            }
            // committed members: reads, results, timestamps
            for (uint32_t j = L.lig; j < nu; j += L.G) {
                const uint32_t m = S.mof[j];
                if (won >> m & 1) a.reads[S.mfirst[m] + (j - S.moff[m])] = S.oldv[j];
            }
            for (uint32_t m = L.lig; m < nmem; m += L.G) {
                if (!(won >> m & 1)) continue;
                const unsigned long long ts = tbase + __popc(taken & ((1u << m) - 1u));
                a.results[S.mt[m]] = gcc_txn_result{GCC_TXN_COMMITTED, S.matt[m], ~0ull};
                a.order_key[S.mt[m]] = ts;
                ++c.commits;
                if (S.matt[m] > c.max_att) c.max_att = S.matt[m];
            }
            const uint32_t lost = pend & ~won;
            if (L.lig == 0) c.aborts += __popc(lost);
            pend = lost;
            if (pend) {
                const uint64_t t2 = __shfl_sync(L.gmask, globaltimer(), L.gbase);
                const uint32_t flag = uatt >= a.max_attempts ? GCC_DEVERR_ATTEMPTS
                                      : t2 > deadline        ? GCC_DEVERR_DEADLINE
                                                             : 0u;
                if (flag) {
                    for (uint32_t m = L.lig; m < nmem; m += L.G) {
                        if (!(pend >> m & 1)) continue;
                        a.results[S.mt[m]] = gcc_txn_result{GCC_TXN_TIMEOUT, S.matt[m], ~0ull};
                        a.order_key[S.mt[m]] = ~0ull;
                        ++c.timeouts;
                        if (S.matt[m] > c.max_att) c.max_att = S.matt[m];
                    }
                    if (L.lig == 0) atomicOr(&a.st->error, flag);
                    pend = 0;
                } else {
                    wake = t2 + backoff_ns(a, S.mt[__ffs(pend) - 1], uatt);
                    if (a.rq && crec != NO_CC && uatt >= a.queue_after) pq = queue_of(a, crec);
                }
            }
            if (!pend) has = false;
            __syncwarp(L.gmask);
        }
        // 3. a warp where nobody attempted this round sleeps until its
        // earliest wake-up (32 ns .. 1 us)
        if (!__any_sync(0xffffffffu, go)) {
            const uint64_t t1 = globaltimer();
            uint32_t rel = 1000;
            if (has && wake > t1) rel = wake - t1 < 1000 ? (uint32_t)(wake - t1) : 1000u;
            else if (has || !finished) rel = 32;
            rel = __reduce_min_sync(0xffffffffu, rel);
            __nanosleep(rel < 32 ? 32 : rel);
        }
    }
}

template <class Work>
__global__ void __launch_bounds__(1024) occ_group_kernel(const __grid_constant__ ExecArgs a) {
    Lane L;
    L.G = a.lanes;
    L.lane = threadIdx.x & 31;
    L.lig = L.lane & (L.G - 1);
    L.gbase = L.lane & ~(L.G - 1);
    L.gmask = (L.G == 32) ? 0xffffffffu : (((1u << L.G) - 1u) << L.gbase);
    UnitStage S;
    setup_unit_stage(a, L, S);
    const uint64_t deadline = __shfl_sync(0xffffffffu, globaltimer(), 0) + a.deadline_ns;
    Counters c;
    SingleFetch<4u> F{&a};
    unit_loop<SingleFetch<4u>, Work>(F, L, S, deadline, c);
    c.atomics += L.n_atom;
    flush_counters(a.st, c);
}

}  // namespace gcc
