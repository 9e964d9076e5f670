// engine.cuh -- internal declarations of the concurrency-control engine.
//
// Memory-ordering primitives, the per-batch device state, kernel argument
// blocks and the host-side launch entry points shared by the translation
// units of the library.  Not part of the public ABI (include/gcc_gb300.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gcc_gb300.h"

namespace gcc {

// ---------------------------------------------------------------------------
// concurrency-control word layouts (one 64-bit word per record, Table II)
// ---------------------------------------------------------------------------
// OCC: bit 63 lock, bits 0..62 version = commit timestamp + 1 (Sec. III-E.2,
// "lock bit : 1, ts : 63").
constexpr uint64_t OCC_LOCK = 1ull << 63;
// 2PL: bit 63 exclusive, bits 32..62 shared-holder count, bits 0..31 exclusive
// holder (transaction id + 1) -- Table II's shared bit / holder count / holder.
constexpr uint64_t TPL_X = 1ull << 63;
constexpr uint64_t TPL_S_ONE = 1ull << 32;
// TO: one 16-byte word per record, updated with a 128-bit CAS: lo = RTS,
// hi = WTS (bits 0..62) | dirty (bit 63, the commit bit of Table II).  Table
// II packs commit bit + 31-bit RTS + 31-bit WTS into 8 bytes, which overflows
// after 2^31 attempts; 64-bit timestamps from a persistent clock never do.
constexpr uint64_t TO_DIRTY = 1ull << 63;
// TicToc: one 16-byte word per record: lo = rts, hi = wts (bits 0..62) | lock
// (bit 63).  The record's current version is valid over [wts, rts]; a commit
// at timestamp c publishes wts = rts = c.
constexpr uint64_t TT_LOCK = 1ull << 63;
// MVCC (multi-version TO): one 16-byte head word per record, 32-bit fields
// with batch-relative timestamps: lo = wts (the record's newest committed
// version) | rts << 32 (its read timestamp), hi = pending writer's timestamp
// (0: none; bits 32..63 unused).  Updated only by 128-bit CAS; read by
// 128-bit loads.  Each (record, field) slot also has a version pointer:
// index + 1 of its newest entry in the batch's version store (0: the table
// slot is its only version).
__host__ __device__ __forceinline__ uint32_t mv_lo(uint64_t w) { return (uint32_t)w; }
__host__ __device__ __forceinline__ uint32_t mv_hi(uint64_t w) { return (uint32_t)(w >> 32); }
__host__ __device__ __forceinline__ uint64_t mv_pack(uint32_t lo, uint32_t hi) {
    return (uint64_t)lo | ((uint64_t)hi << 32);
}
// DET: bits 32..63 ops completed on the record, bits 0..31 writes completed,
// both counted from the record's first position in the batch's sorted
// access table (Sec. III-E.3, "access tables").
constexpr uint64_t DET_READ_DONE = 1ull << 32;
constexpr uint64_t DET_WRITE_DONE = (1ull << 32) + 1;

// Per-batch device state (zeroed by the batch-begin kernel).
struct BatchState {
    unsigned long long fetch;        // next transaction id to hand out
    unsigned long long ticket;       // 2PL commit counter
    unsigned long long ticket_base;  // OCC/TO: persistent clock at batch start
    unsigned long long committed;
    unsigned long long aborts;
    unsigned long long timeouts;
    unsigned long long invalid;
    unsigned long long max_attempts;
    unsigned long long atomics;      // global atomic operations of the execute kernel
    unsigned long long mv_used;      // MVCC: version-store entries taken
    unsigned int error;              // GCC_DEVERR_* bits
    unsigned int pad;
};

// Retry queues per database (one 64-bit word each).
constexpr uint32_t RETRY_QUEUES = 1u << 16;

// Persistent per-database device state.
struct DbState {
    unsigned long long occ_clock;    // OCC commit timestamps, never reset
    unsigned long long to_clock;     // TO attempt timestamps, never reset
};

// ---------------------------------------------------------------------------
// PTX memory-order helpers (gpu scope)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 16-byte record slot access (one vector transaction).
__device__ __forceinline__ ulonglong2 ld_slot16(const void* p) {
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
                 : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_slot16(void* p, ulonglong2 v) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};"
                 ::"l"(p), "l"(v.x), "l"(v.y) : "memory");
}
// 16-byte load as one 128-bit access, with acquire semantics (a record's
// MVCC head word: its four fields are read together).
__device__ __forceinline__ ulonglong2 ld128_acquire(const void* p) {
    ulonglong2 v;
    asm volatile(
        "{\n\t.reg .b128 d;\n\t"
        "ld.acquire.gpu.global.b128 d, [%2];\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// 16-byte compare-and-swap (sm_90 and later): both halves compared and
// replaced as one atomic operation.
__device__ __forceinline__ ulonglong2 cas128(ulonglong2* p, ulonglong2 cmp, ulonglong2 val) {
    ulonglong2 old;
    asm volatile(
        "{\n\t.reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.relaxed.gpu.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old.x), "=l"(old.y)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
        : "memory");
    return old;
}
__device__ __forceinline__ uint64_t cas64(uint64_t* p, uint64_t cmp, uint64_t val) {
    return atomicCAS(reinterpret_cast<unsigned long long*>(p), cmp, val);
}
// Lock acquisitions: acquire semantics order the caller's later accesses
// (the locked record's value) after the CAS.
__device__ __forceinline__ uint64_t cas64_acquire(uint64_t* p, uint64_t cmp, uint64_t val) {
    uint64_t old;
    asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;"
                 : "=l"(old) : "l"(p), "l"(cmp), "l"(val) : "memory");
    return old;
}
__device__ __forceinline__ ulonglong2 cas128_acquire(ulonglong2* p, ulonglong2 cmp, ulonglong2 val) {
    ulonglong2 old;
    asm volatile(
        "{\n\t.reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.acquire.gpu.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old.x), "=l"(old.y)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
        : "memory");
    return old;
}
// Lock releases and done-counters: release semantics order the caller's
// earlier accesses before the update.
__device__ __forceinline__ uint64_t add64_release(uint64_t* p, uint64_t v) {
    uint64_t old;
    asm volatile("atom.release.gpu.global.add.u64 %0, [%1], %2;"
                 : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint64_t max64(uint64_t* p, uint64_t v) {
    return atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ uint64_t add64(uint64_t* p, uint64_t v) {
    return atomicAdd(reinterpret_cast<unsigned long long*>(p), v);
}
// Release/acquire fence at gpu scope.  Every ordering the schemes rely on is
// release/acquire through an atomic on a shared location (a lock CAS, the
// commit clock, a done counter), which this fence provides without the cost
// of a sequentially consistent one.
__device__ __forceinline__ void fence_acq_rel() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One ticket from a counter per calling lane, with one atomic per warp and
// counter: the lanes active at the call that name the same counter share a
// single atomicAdd (lanes of one warp may name different counters -- in the
// batched form, groups of one warp work on different databases).  *n_atom
// (when given) counts the atomic on the lane that issues it.
__device__ __forceinline__ unsigned long long agg_ticket(unsigned long long* ctr,
                                                        unsigned step = 1,
                                                        uint32_t* n_atom = nullptr) {
    const unsigned mask = __match_any_sync(__activemask(), reinterpret_cast<uintptr_t>(ctr));
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == leader) {
        base = atomicAdd(ctr, (unsigned long long)__popc(mask) * step);
        if (n_atom) ++*n_atom;
    }
    base = __shfl_sync(mask, base, leader);
    return base + (unsigned long long)__popc(mask & lanemask_lt()) * step;
}
// The same with an acquire-release atomic: the caller's earlier memory
// operations are ordered before its ticket and its later ones after it, so a
// thread whose ticket follows this one (the counter's read-modify-write chain
// carries the release) also sees everything that preceded this ticket.
__device__ __forceinline__ unsigned long long agg_ticket_acq_rel(unsigned long long* ctr,
                                                                uint32_t* n_atom = nullptr) {
    const unsigned mask = __match_any_sync(__activemask(), reinterpret_cast<uintptr_t>(ctr));
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == leader) {
        const unsigned long long inc = (unsigned long long)__popc(mask);
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
                     : "=l"(base) : "l"(ctr), "l"(inc) : "memory");
        if (n_atom) ++*n_atom;
    }
    base = __shfl_sync(mask, base, leader);
    return base + (unsigned long long)__popc(mask & lanemask_lt());
}

// 64-bit mixing (splitmix64 finaliser) for jitter and abort injection.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27; z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Op kinds that modify their record (the deterministic scheme's writers).
__host__ __device__ __forceinline__ bool kind_writes(uint32_t kind) {
    switch (kind) {
        case GCC_OP_ADD:
        case GCC_OE_W_PAY:
        case GCC_OE_D_NEWORDER:
        case GCC_OE_D_PAY:
        case GCC_OE_C_PAY:
        case GCC_OE_S_NEWORDER:
        case GCC_OE_C_PAY_BY_NAME:
            return true;
        default:
            return false;
    }
}

// Concurrency-control record of an op: the key itself for key-value tables;
// for order-entry, the row offset by its table's base in the record space
// (warehouse, district, customer, stock).  Item reads need no control and
// map to `none`.
__host__ __device__ __forceinline__ uint32_t cc_record(uint64_t d, int schema, uint32_t W,
                                                       uint32_t none) {
    const uint32_t key = (uint32_t)d;
    if (schema == GCC_SCHEMA_KV) return key;
    switch ((uint32_t)(d >> 40) & 0xffu) {
        case GCC_OE_W_READ: case GCC_OE_W_PAY: return key < W ? key : none;
        case GCC_OE_D_NEWORDER: case GCC_OE_D_PAY: return key < 10u * W ? W + key : none;
        case GCC_OE_C_READ: case GCC_OE_C_PAY: return key < 30000u * W ? 11u * W + key : none;
        case GCC_OE_S_NEWORDER: return key < 100000u * W ? 30011u * W + key : none;
        default: return none;
    }
}

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
struct ExecArgs {
    // batch
    const gcc_txn* txns;
    const uint64_t* ops;          // gcc_op as packed 64-bit words
    const ulonglong2* operands;
    uint32_t n_txns;
    uint64_t n_ops;
    gcc_txn_result* results;
    ulonglong2* reads;
    // database
    uint8_t* table;               // key-value slots (field-major)
    uint64_t n_records;
    uint32_t n_fields;
    uint64_t* meta;               // one concurrency-control word per record
    uint64_t n_meta;
    int64_t* const* cols;         // order-entry columns (device array of pointers)
    uint32_t n_warehouses;
    uint32_t order_cap;
    // scheme scratch
    const uint32_t* need;         // DET: per-op wait threshold
    unsigned long long* order_key;// OCC/TO/TicToc: raw commit timestamp per txn
    uint32_t* seq;                // TicToc: commit sequence number per txn (ties)
    uint32_t det_all;             // DET dataflow: every access waits for all earlier ones
    int order_key_uses_base;      // OCC: timestamps count from BatchState::ticket_base
    BatchState* st;
    DbState* dbs;
    // policy
    uint32_t lanes;               // lanes per transaction (power of two <= 32)
    uint32_t max_ops;             // staging capacity per transaction
    uint32_t collapse;
    uint32_t backoff_base_ns;
    uint32_t backoff_cap_ns;
    uint32_t max_attempts;
    uint32_t read_retries;
    uint32_t inject_ppm;
    uint64_t wait_budget_ns;
    uint64_t deadline_ns;
    uint64_t seed;
    uint64_t* rq;               // retry queues (null: randomized backoff only)
    uint32_t rq_mask;           // queues - 1 (a power of two)
    uint32_t queue_turn_ns;     // estimated time per queue turn
    uint32_t queue_width;       // tickets a queue admits at once
    uint32_t queue_after;       // aborts before a transaction uses the queues
    // MVCC version store of the batch: entry i = (wts, next, record, field,
    // value); capacity n_ops (one entry per committed write)
    uint32_t* mv_wts;
    uint32_t* mv_next;           // index + 1 of the slot's previous entry, 0: none
    uint32_t* mv_rec;
    uint32_t* mv_field;
    ulonglong2* mv_val;
    uint32_t* mv_slot;           // per slot (field-major): its newest entry + 1
    // OCC group commit (key-value): units of up to group_u transactions
    const uint32_t* unit_link;   // per txn: next member | follower bit (null: off)
    uint32_t group_u;
};


// Shared-memory staging per op: descriptor, observed word, value read, value
// to write and one more word (TicToc's rts): the read and write sets live in
// shared memory while the transaction runs, so aborted attempts never touch
// the output arrays.
constexpr uint32_t STAGE_BYTES_PER_OP = 8 + 8 + 16 + 16 + 8;

// ---------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------
// Key-value execute kernel for one scheme and slot width.
cudaError_t launch_kv_exec(gcc_scheme scheme, uint32_t field_bytes, const ExecArgs& a,
                           int grid, int block, size_t smem, cudaStream_t s);
int kv_exec_occupancy(gcc_scheme scheme, uint32_t field_bytes, int block, size_t smem);
// OCC with group commit on key-value batches (occ_group.cu): unit formation,
// staging bytes per lane group, launcher and occupancy.
struct SortScratch;
cudaError_t occ_form_units(const ExecArgs& a, uint32_t* cnt, SortScratch& s, uint32_t* link,
                           uint32_t U, uint32_t min_writes, cudaStream_t st);
uint32_t occ_form_units_launches(uint64_t n_records);
size_t occ_group_stage_bytes(uint32_t U, uint32_t max_ops);
cudaError_t launch_kv_occ_group(uint32_t field_bytes, const ExecArgs& a, int grid, int block,
                                size_t smem, cudaStream_t s);
int kv_occ_group_occupancy(uint32_t field_bytes, int block, size_t smem);
// Order-entry execute kernel for one scheme.
cudaError_t launch_oe_exec(gcc_scheme scheme, const ExecArgs& a, int grid, int block,
                           size_t smem, cudaStream_t s);
int oe_exec_occupancy(gcc_scheme scheme, int block, size_t smem);

// Batch begin: zero the state; OCC: record the clock as ticket base.
cudaError_t launch_batch_begin(BatchState* st, DbState* dbs, gcc_scheme scheme,
                               cudaStream_t s);

// Stable LSD radix sort of (key, value) u32 pairs on the low `bits` bits.
// Sorted output lands in (*keys_out, *vals_out), one of the two buffer pairs.
struct SortScratch {
    uint32_t *k0, *v0, *k1, *v1;
    uint32_t* hist;               // 256 * max_tiles
    uint32_t* totals;             // 256
    size_t max_items;
};
size_t sort_max_tiles(size_t n);
cudaError_t radix_sort_pairs(SortScratch& s, size_t n, int bits, uint32_t** keys_out,
                             uint32_t** vals_out, cudaStream_t st);

// Exclusive prefix sum of u32 (in place), with `tmp` of >= scan_tmp_words(n).
size_t scan_tmp_words(size_t n);
cudaError_t exclusive_scan_u32(uint32_t* data, size_t n, uint32_t* tmp, cudaStream_t st);

// Deterministic-scheme preprocessing: access table (record, op) sorted by
// record then transaction id, per-op wait thresholds and per-record counters.
struct DetPrep {
    const uint64_t* ops;
    uint64_t n_ops;
    uint64_t* meta;
    uint32_t* need;
    const uint32_t* op_cc_key;    // optional: concurrency-control record per op
};
cudaError_t det_prepare(const ExecArgs& a, SortScratch& s, uint32_t* scan_tmp, int key_bits,
                        int schema, cudaStream_t st, bool all_conflict = false);

// Record `msg` as this thread's gcc_last_error() and return `s`.
gcc_status set_error(gcc_status s, const char* msg);

// Deterministic scheme on a key-value batch by segmented prefix sums; `flags`
// holds 2 * n_txns words, `seg_tmp` fold_seg_bytes(n_ops) bytes.
size_t fold_seg_bytes(size_t max_ops);
// Deterministic order-entry batch: each record's accesses applied in id order
// by one warp over the sorted access table (reads, final records, NewOrder
// inserts, results, dense ranks, batch counters).  `flags` holds 2 * n_txns
// words, `heads` n_ops words; key_bits covers n_meta.
cudaError_t det_serial_oe(const ExecArgs& a, SortScratch& s, uint32_t* scan_tmp, uint32_t* flags,
                          uint32_t* heads, int key_bits, int sm_count, cudaStream_t st);
int det_serial_oe_launches(int key_bits);
cudaError_t det_fold_kv(const ExecArgs& a, uint32_t field_bytes, SortScratch& s,
                        uint32_t* scan_tmp, uint32_t* flags, void* seg_tmp, cudaStream_t st);

// OCC / TO: replace raw commit timestamps by dense ranks 0..committed-1.
cudaError_t densify_commit_order(const ExecArgs& a, SortScratch& s, cudaStream_t st);
// Deterministic scheme run op by op: dense ranks in transaction-id order over
// the committed transactions (`flags`: n_txns words, `scan_tmp`:
// scan_tmp_words(n_txns) words).
cudaError_t densify_in_id_order(const ExecArgs& a, uint32_t* flags, uint32_t* scan_tmp,
                                cudaStream_t st);
// TicToc: dense ranks in (timestamp, sequence number) order.
cudaError_t densify_tictoc(const ExecArgs& a, SortScratch& s, cudaStream_t st);
// Payment by last name: per-district index of the customers in (last name,
// first name, index) order (idx: customer numbers, last_sorted: their last
// names; 3000 entries per district), and the batch's ops with every by-name
// payment op replaced by a payment of the customer it names (or by an op of
// unknown kind, which makes its transaction invalid, when nobody has the
// name).
cudaError_t build_name_index(const int64_t* c_last, const int64_t* c_first, uint32_t n_districts,
                             uint32_t* idx, int64_t* last_sorted, cudaStream_t st);
cudaError_t resolve_by_name(const uint64_t* ops, uint64_t n, uint32_t W, const uint32_t* idx,
                            const int64_t* last_sorted, uint64_t* out, cudaStream_t st);
// MVCC, after the execute kernel: every slot's newest entry written into the
// table, its version pointer cleared, every head word zeroed.
cudaError_t launch_mv_flatten(const ExecArgs& a, uint32_t field_bytes, cudaStream_t st);
// Seeded initial values of a key-value table, written on the device.
cudaError_t launch_seeded_init(uint8_t* table, uint64_t n_records, uint32_t n_fields,
                               uint32_t field_bytes, uint64_t seed, int sm_count,
                               cudaStream_t st);

}  // namespace gcc
