// api.cu -- host runtime behind the C ABI in include/gcc_gb300.h.
//
// Owns the database's device memory (tables, one concurrency-control word per
// record, batch scratch), decides when the control words must be reset
// between batches, sizes the persistent grid from the occupancy of the
// chosen kernel, and runs a batch as a stream-ordered sequence:
//   batch-begin -> [deterministic: access table, sort, thresholds]
//   -> execute kernel -> [OCC/TO: dense commit ranks].
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "runtime.cuh"

namespace {
thread_local std::string g_err;
}  // namespace

namespace gcc {
namespace rt {
gcc_status fail(gcc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define GCC_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(e_ == cudaErrorMemoryAllocation ? GCC_ERR_NOMEM : GCC_ERR_CUDA, \
                        "%s failed: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

}  // namespace rt
}  // namespace gcc

using gcc::rt::fail;
using gcc::rt::OE_NCOLS;
using gcc::rt::oe_rows;


namespace gcc {
namespace rt {

gcc_exec_params defaults() {
    gcc_exec_params p{};
    p.lanes_per_txn = 16;
    p.warps_per_block = 8;
    p.blocks_per_sm = 0;
    p.collapse = 1;
    p.backoff_base_ns = 128;
    p.backoff_cap_ns = 1000000;
    p.max_attempts = 1u << 24;
    p.read_retries = 8;
    p.wait_budget_ns = 2000000000ull;
    p.deadline_ns = 60000000000ull;
    p.seed = 0x5EEDull;
    p.inject_abort_ppm = 0;
    p.retry_queue = 1;
    p.queue_turn_ns = 1000;
    p.queue_width = 1;
    p.queue_after = 0;                   // per scheme, see queue_after_for
    p.group_commit = 1;
    p.group_min_writes = 32;
    return p;
}

uint32_t queue_after_for(const gcc_exec_params& p, gcc_scheme scheme) {
    if (p.queue_after) return p.queue_after;
    return scheme == GCC_OCC ? 64u : 16u;
}

gcc_exec_params merged(const gcc_exec_params* in) {
    gcc_exec_params p = defaults();
    if (!in) return p;
    if (in->lanes_per_txn) p.lanes_per_txn = in->lanes_per_txn;
    if (in->warps_per_block) p.warps_per_block = in->warps_per_block;
    p.blocks_per_sm = in->blocks_per_sm;
    if (in->collapse) p.collapse = in->collapse;
    if (in->backoff_base_ns) p.backoff_base_ns = in->backoff_base_ns;
    if (in->backoff_cap_ns) p.backoff_cap_ns = in->backoff_cap_ns;
    p.immediate_restart = in->immediate_restart;
    if (in->max_attempts) p.max_attempts = in->max_attempts;
    if (in->read_retries) p.read_retries = in->read_retries;
    if (in->wait_budget_ns) p.wait_budget_ns = in->wait_budget_ns;
    if (in->deadline_ns) p.deadline_ns = in->deadline_ns;
    if (in->seed) p.seed = in->seed;
    p.inject_abort_ppm = in->inject_abort_ppm;
    p.det_dataflow = in->det_dataflow;
    if (in->retry_queue) p.retry_queue = in->retry_queue;
    if (in->queue_turn_ns) p.queue_turn_ns = in->queue_turn_ns;
    if (in->queue_width) p.queue_width = in->queue_width;
    if (in->queue_after) p.queue_after = in->queue_after;
    if (in->group_commit) p.group_commit = in->group_commit;
    if (in->group_min_writes) p.group_min_writes = in->group_min_writes;
    return p;
}

int bit_length(uint64_t v) {
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

template <class T>
gcc_status dev_alloc(T** p, uint64_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return GCC_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(GCC_ERR_NOMEM, "cudaMalloc of %llu bytes for %s failed: %s",
                    (unsigned long long)bytes, what, cudaGetErrorString(e));
    }
    e = cudaMemset(*p, 0, bytes);
    if (e != cudaSuccess) return fail(GCC_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
    return GCC_OK;
}

void free_db(gcc_db* db) {
    cudaSetDevice(db->d.device);
    if (db->stream) cudaStreamSynchronize(db->stream);
    cudaFree(db->table);
    for (auto& c : db->cols) cudaFree(c);
    cudaFree(db->d_cols);
    cudaFree(db->meta);
    cudaFree(db->st);
    cudaFree(db->dbs);
    cudaFree(db->rq);
    cudaFree(db->sort.k0);
    cudaFree(db->sort.v0);
    cudaFree(db->sort.k1);
    cudaFree(db->sort.v1);
    cudaFree(db->sort.hist);
    cudaFree(db->sort.totals);
    cudaFree(db->scan_tmp);
    cudaFree(db->need);
    cudaFree(db->order_key);
    cudaFree(db->fold_flags);
    cudaFree(db->fold_seg);
    cudaFree(db->mv_slot);
    cudaFree(db->unit_cnt);
    cudaFree(db->unit_link);
    cudaFree(db->name_idx);
    cudaFree(db->name_last);
    cudaFree(db->ops_resolved);
    if (db->h_states) cudaFreeHost(db->h_states);
    for (auto& r : db->stages)
        for (auto& e : r.ev)
            if (e) cudaEventDestroy(e);
    if (db->stream) cudaStreamDestroy(db->stream);
    delete db;
}

gcc_status create_impl(const gcc_db_desc* desc, gcc_db** out) {
    if (!desc || !out) return fail(GCC_ERR_INVALID, "null argument");
    *out = nullptr;
    const gcc_db_desc& d = *desc;
    if (d.schema == GCC_SCHEMA_KV) {
        if (d.field_bytes != 8 && d.field_bytes != 16)
            return fail(GCC_ERR_INVALID, "field_bytes must be 8 or 16");
        if (d.n_records == 0 || d.n_records > (1ull << 31))
            return fail(GCC_ERR_INVALID, "n_records must be in 1..2^31");
        if (d.n_fields == 0 || d.n_fields > 255)
            return fail(GCC_ERR_INVALID, "n_fields must be in 1..255");
    } else if (d.schema == GCC_SCHEMA_ORDER_ENTRY) {
        if (d.n_warehouses == 0 || d.n_warehouses > 1024)
            return fail(GCC_ERR_INVALID, "n_warehouses must be in 1..1024");
        if (d.order_cap < 3000 || d.order_cap > (1u << 24))
            return fail(GCC_ERR_INVALID, "order_cap must be in 3000..2^24");
    } else {
        return fail(GCC_ERR_INVALID, "unknown schema %u", d.schema);
    }
    if (d.max_ops_per_txn == 0 || d.max_ops_per_txn > 64)
        return fail(GCC_ERR_INVALID, "max_ops_per_txn must be in 1..64");
    if (d.max_batch_txns == 0 || d.max_batch_txns > (1ull << 31))
        return fail(GCC_ERR_INVALID, "max_batch_txns must be in 1..2^31");
    if (d.max_batch_ops == 0 || d.max_batch_ops >= (1ull << 32))
        return fail(GCC_ERR_INVALID, "max_batch_ops must be in 1..2^32-1");
    int ndev = 0;
    GCC_CK(cudaGetDeviceCount(&ndev));
    if (d.device < 0 || d.device >= ndev) return fail(GCC_ERR_INVALID, "no CUDA device %d", d.device);
    GCC_CK(cudaSetDevice(d.device));

    gcc_db* db = new (std::nothrow) gcc_db();
    if (!db) return fail(GCC_ERR_NOMEM, "host allocation failed");
    db->d = d;
    gcc_status s = GCC_OK;
    auto bail = [&](gcc_status st) { free_db(db); return st; };
    if (cudaDeviceGetAttribute(&db->sm_count, cudaDevAttrMultiProcessorCount, d.device) != cudaSuccess)
        return bail(fail(GCC_ERR_CUDA, "cannot query SM count"));
    if (cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(GCC_ERR_CUDA, "cannot create stream"));

    if (d.schema == GCC_SCHEMA_KV) {
        db->table_bytes = d.n_records * d.n_fields * d.field_bytes;
        if ((s = dev_alloc(&db->table, db->table_bytes, "table"))) return bail(s);
        db->n_meta = d.n_records;
    } else {
        const uint64_t W = d.n_warehouses;
        for (int c = 0; c < OE_NCOLS; ++c) {
            db->col_bytes[c] = oe_rows(c, W, d.order_cap) * sizeof(int64_t);
            if ((s = dev_alloc(&db->cols[c], db->col_bytes[c], "order-entry column"))) return bail(s);
        }
        if ((s = dev_alloc(&db->d_cols, sizeof(int64_t*) * OE_NCOLS, "column table"))) return bail(s);
        if (cudaMemcpy(db->d_cols, db->cols, sizeof(int64_t*) * OE_NCOLS, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return bail(fail(GCC_ERR_CUDA, "cannot upload column table"));
        db->n_meta = W * (1 + OE_DIST + OE_DIST * OE_CUST) + W * OE_ITEMS;
        const uint64_t n_cust = W * OE_DIST * OE_CUST;
        if ((s = dev_alloc(&db->name_idx, n_cust * 4, "last-name index"))) return bail(s);
        if ((s = dev_alloc(&db->name_last, n_cust * 8, "last-name index"))) return bail(s);
        if ((s = dev_alloc(&db->ops_resolved, d.max_batch_ops * 8, "resolved ops"))) return bail(s);
        if (gcc::build_name_index(db->cols[gcc::rt::OE_C_LAST], db->cols[gcc::rt::OE_C_FIRST],
                                  (uint32_t)(W * OE_DIST), db->name_idx, db->name_last,
                                  db->stream) != cudaSuccess ||
            cudaStreamSynchronize(db->stream) != cudaSuccess)
            return bail(fail(GCC_ERR_CUDA, "cannot build the last-name index"));
    }
    if ((s = dev_alloc(&db->meta, db->n_meta * 16, "control words (16 bytes per record for TO)"))) return bail(s);
    if ((s = dev_alloc(&db->st, sizeof(gcc::BatchState), "batch state"))) return bail(s);
    if ((s = dev_alloc(&db->dbs, sizeof(gcc::DbState), "db state"))) return bail(s);
    if ((s = dev_alloc(&db->rq, (uint64_t)gcc::RETRY_QUEUES * 8, "retry queues"))) return bail(s);
    const uint64_t items = std::max<uint64_t>(d.max_batch_ops, d.max_batch_txns);
    db->sort.max_items = items;
    if ((s = dev_alloc(&db->sort.k0, items * 4, "sort keys"))) return bail(s);
    if ((s = dev_alloc(&db->sort.v0, items * 4, "sort values"))) return bail(s);
    if ((s = dev_alloc(&db->sort.k1, items * 4, "sort keys"))) return bail(s);
    if ((s = dev_alloc(&db->sort.v1, items * 4, "sort values"))) return bail(s);
    if ((s = dev_alloc(&db->sort.hist, gcc::sort_max_tiles(items) * 256 * 4, "sort histogram")))
        return bail(s);
    if ((s = dev_alloc(&db->sort.totals, 256 * 4, "sort totals"))) return bail(s);
    if ((s = dev_alloc(&db->scan_tmp, gcc::scan_tmp_words(items) * 4, "scan scratch"))) return bail(s);
    if ((s = dev_alloc(&db->need, d.max_batch_ops * 4, "wait thresholds"))) return bail(s);
    if ((s = dev_alloc(&db->order_key, d.max_batch_txns * 8, "commit keys"))) return bail(s);
    if ((s = dev_alloc(&db->fold_flags, d.max_batch_txns * 8, "validity flags and ranks")))
        return bail(s);
    if (d.schema == GCC_SCHEMA_KV &&
        (s = dev_alloc(&db->fold_seg, gcc::fold_seg_bytes(d.max_batch_ops), "fold carries")))
        return bail(s);
    // MVCC version pointers, one per slot, zero between batches
    if (d.schema == GCC_SCHEMA_KV &&
        (s = dev_alloc(&db->mv_slot, d.n_records * d.n_fields * 4, "version pointers")))
        return bail(s);
    // OCC group commit: write counts per record and a link word per transaction
    if (d.schema == GCC_SCHEMA_KV && d.n_records < 0xffffffffull &&
        ((s = dev_alloc(&db->unit_cnt, d.n_records * 4, "group-commit write counts")) ||
         (s = dev_alloc(&db->unit_link, d.max_batch_txns * 4, "group-commit links"))))
        return bail(s);
    db->n_h_states = GCC_MAX_OUTSTANDING_BATCHES;
    if (cudaMallocHost(&db->h_states, sizeof(gcc::BatchState) * db->n_h_states) != cudaSuccess)
        return bail(fail(GCC_ERR_NOMEM, "cannot allocate pinned batch states"));
    for (uint32_t i = db->n_h_states; i > 0; --i) db->free_h_states.push_back(i - 1);
    for (auto& r : db->stages)
        for (auto& e : r.ev)
            if (cudaEventCreate(&e) != cudaSuccess)
                return bail(fail(GCC_ERR_CUDA, "cannot create timing events"));
    *out = db;
    return GCC_OK;
}

gcc_status validate_params(const gcc_exec_params& p) {
    const uint32_t g = p.lanes_per_txn;
    if (g == 0 || g > 32 || (g & (g - 1)))
        return fail(GCC_ERR_INVALID, "lanes_per_txn must be a power of two in 1..32");
    if (p.warps_per_block == 0 || p.warps_per_block > 32)
        return fail(GCC_ERR_INVALID, "warps_per_block must be in 1..32");
    if (p.collapse > 2) return fail(GCC_ERR_INVALID, "collapse must be 0, 1 or 2");
    if (p.group_commit > 8) return fail(GCC_ERR_INVALID, "group_commit must be in 0..8");
    if (p.retry_queue > 2) return fail(GCC_ERR_INVALID, "retry_queue must be 0, 1 or 2");
    if (p.det_dataflow > 2) return fail(GCC_ERR_INVALID, "det_dataflow must be 0, 1 or 2");
    return GCC_OK;
}

gcc_status prepare_meta(gcc_db* db, gcc_scheme scheme, cudaStream_t st) {
    // control words: reset whenever the previous batch left them in a state
    // the scheme cannot start from
    bool reset = false;
    switch (scheme) {
        case GCC_NO_WAIT_2PL:
        case GCC_2PL_WAIT_DIE: reset = db->meta_state != META_ZERO; break;
        case GCC_OCC: reset = db->meta_state != META_ZERO && db->meta_state != META_OCC; break;
        case GCC_TO: reset = db->meta_state != META_ZERO && db->meta_state != META_TO; break;
        case GCC_DET: reset = false; break;    // per-record counters set by preprocessing
        case GCC_TICTOC:
            reset = db->meta_state != META_ZERO && db->meta_state != META_TICTOC;
            break;
        case GCC_MVCC: reset = db->meta_state != META_ZERO; break;   // empty heads
    }
    if (reset) GCC_CK(cudaMemsetAsync(db->meta, 0, db->n_meta * 16, st));
    return GCC_OK;
}

gcc_status execute_impl(gcc_db* db, gcc_scheme scheme, const gcc_txn* d_txns, uint32_t n_txns,
                        const gcc_op* d_ops, const gcc_operand* d_operands, uint64_t n_ops,
                        const gcc_exec_params* params, gcc_txn_result* d_results,
                        gcc_operand* d_reads, cudaStream_t stream) {
    if (!db) return fail(GCC_ERR_INVALID, "null database");
    if ((unsigned)scheme > GCC_MVCC)
        return fail(GCC_ERR_INVALID, "unknown scheme %d", (int)scheme);
    if (scheme == GCC_MVCC && db->d.schema != GCC_SCHEMA_KV)
        return fail(GCC_ERR_INVALID, "GCC_MVCC runs key-value databases only");
    if (n_txns > db->d.max_batch_txns || n_ops > db->d.max_batch_ops)
        return fail(GCC_ERR_CAPACITY, "batch of %u txns / %llu ops exceeds the database maxima",
                    n_txns, (unsigned long long)n_ops);
    if (n_txns && (!d_txns || !d_results)) return fail(GCC_ERR_INVALID, "null batch pointer");
    if (n_ops && (!d_ops || !d_operands || !d_reads)) return fail(GCC_ERR_INVALID, "null op pointer");
    gcc_exec_params p = merged(params);
    gcc_status s = validate_params(p);
    if (s) return s;
    // the prefix-sum evaluation sorts 32-bit slot ids, one id past the last
    // slot marking invalid transactions' accesses
    if (scheme == GCC_DET && db->d.schema == GCC_SCHEMA_KV && !p.det_dataflow &&
        (uint64_t)db->d.n_fields * db->d.n_records >= (1ull << 32))
        return fail(GCC_ERR_CAPACITY,
                    "deterministic key-value batches by prefix sums need n_records * n_fields "
                    "below 2^32 (det_dataflow = 1 has no such limit)");
    GCC_CK(cudaSetDevice(db->d.device));
    cudaStream_t st = stream ? stream : db->stream;
    StageRec& rec = db->stages[db->n_stages % STAGE_RING];
    GCC_CK(cudaEventRecord(rec.ev[0], st));
    uint32_t launches = 0;

    if ((s = prepare_meta(db, scheme, st))) return s;

    gcc::ExecArgs a{};
    a.txns = d_txns;
    a.ops = reinterpret_cast<const uint64_t*>(d_ops);
    a.operands = reinterpret_cast<const ulonglong2*>(d_operands);
    a.n_txns = n_txns;
    a.n_ops = n_ops;
    a.results = d_results;
    a.reads = reinterpret_cast<ulonglong2*>(d_reads);
    a.table = db->table;
    a.n_records = db->d.n_records;
    a.n_fields = db->d.n_fields;
    a.meta = db->meta;
    a.n_meta = db->n_meta;
    a.cols = db->d_cols;
    a.n_warehouses = db->d.n_warehouses;
    a.order_cap = db->d.order_cap;
    a.need = db->need;
    a.order_key = db->order_key;
    a.seq = db->fold_flags;
    a.order_key_uses_base = scheme == GCC_OCC || scheme == GCC_TO;   // MVCC: batch-relative
    // MVCC version store: one entry per committed write, in scratch that
    // the commit ranks only need after the store has been flattened
    a.mv_wts = db->sort.k0;
    a.mv_next = db->sort.v0;
    a.mv_field = db->sort.k1;
    a.mv_rec = db->sort.v1;
    a.mv_val = static_cast<ulonglong2*>(db->fold_seg);
    a.mv_slot = db->mv_slot;
    a.st = db->st;
    a.dbs = db->dbs;
    a.lanes = p.lanes_per_txn;
    a.max_ops = db->d.max_ops_per_txn;
    a.collapse = p.collapse;
    a.backoff_base_ns = p.immediate_restart ? 0u : p.backoff_base_ns;
    a.backoff_cap_ns = p.backoff_cap_ns;
    a.max_attempts = p.max_attempts;
    a.read_retries = p.read_retries;
    a.inject_ppm = p.inject_abort_ppm;
    a.wait_budget_ns = p.wait_budget_ns;
    a.deadline_ns = p.deadline_ns;
    a.seed = p.seed;
    a.rq = (p.retry_queue == 2 || p.immediate_restart) ? nullptr : db->rq;
    a.rq_mask = gcc::RETRY_QUEUES - 1;
    a.queue_turn_ns = p.queue_turn_ns;
    a.det_all = p.det_dataflow == 2 ? 1u : 0u;
    a.queue_width = p.queue_width;
    a.queue_after = queue_after_for(p, scheme);

    GCC_CK(gcc::launch_batch_begin(db->st, db->dbs, scheme, st));
    launches += 1;
    const bool kv = db->d.schema == GCC_SCHEMA_KV;
    if (!kv && n_ops) {
        // payments by last name become payments of the customer they name,
        // before any scheme sees the batch
        GCC_CK(gcc::resolve_by_name(a.ops, n_ops, db->d.n_warehouses, db->name_idx, db->name_last,
                                    db->ops_resolved, st));
        a.ops = db->ops_resolved;
        launches += 1;
    }
    // deterministic key-value batches: every record chain by prefix sums
    const bool fold = scheme == GCC_DET && kv && !p.det_dataflow;
    if (fold) {
        GCC_CK(cudaEventRecord(rec.ev[1], st));
        GCC_CK(gcc::det_fold_kv(a, db->d.field_bytes, db->sort, db->scan_tmp, db->fold_flags,
                                db->fold_seg, st));
        const int bits = bit_length((uint64_t)db->d.n_fields * db->d.n_records);
        launches += 2 + 3 * ((bits + 7) / 8) + 4 + 1 + 3 + 2;
        GCC_CK(cudaEventRecord(rec.ev[2], st));
        GCC_CK(cudaEventRecord(rec.ev[3], st));
        rec.stream = st;
        rec.scheme = scheme;
        rec.n_txns = n_txns;
        rec.launches = launches;
        rec.grid = 0;
        rec.used = true;
        db->n_stages++;                  // control words untouched
        db->last_stream = st;
        db->last_scheme = scheme;
        db->last_n_txns = n_txns;
        return GCC_OK;
    }
    // deterministic order-entry batches: every record chain in one pass
    if (scheme == GCC_DET && !kv && !p.det_dataflow) {
        const int bits = std::max(1, bit_length(db->n_meta));
        GCC_CK(cudaEventRecord(rec.ev[1], st));
        GCC_CK(gcc::det_serial_oe(a, db->sort, db->scan_tmp, db->fold_flags, db->need, bits,
                                  db->sm_count, st));
        launches += gcc::det_serial_oe_launches(bits);
        GCC_CK(cudaEventRecord(rec.ev[2], st));
        GCC_CK(cudaEventRecord(rec.ev[3], st));
        rec.stream = st;
        rec.scheme = scheme;
        rec.n_txns = n_txns;
        rec.launches = launches;
        rec.grid = 0;
        rec.used = true;
        db->n_stages++;                  // control words untouched
        db->last_stream = st;
        db->last_scheme = scheme;
        db->last_n_txns = n_txns;
        return GCC_OK;
    }
    if (scheme == GCC_DET && n_ops) {
        // records 0..n_meta-1 plus the key n_meta that marks out-of-range
        // ops: the sort must cover n_meta itself so that those ops sort after
        // every record's run (a power-of-two n_meta needs one more bit)
        const int bits = std::max(1, bit_length(db->n_meta));
        GCC_CK(gcc::det_prepare(a, db->sort, db->scan_tmp, bits, db->d.schema, st,
                                p.det_dataflow == 2));
        launches += 1 + 3 * ((bits + 7) / 8) + 1 + 3 + 1;   // emit, sort, flags, scan, need
    }
    // OCC group commit on key-value batches: units of up to gu transactions
    // (each unit's ops are staged together: at most 255 per unit)
    const uint32_t gu = (scheme == GCC_OCC && kv && db->unit_link && p.group_commit >= 2)
                            ? std::min<uint32_t>(p.group_commit, 255u / db->d.max_ops_per_txn)
                            : 1u;
    if (gu >= 2 && n_txns) {
        a.unit_link = db->unit_link;
        a.group_u = gu;
        GCC_CK(gcc::occ_form_units(a, db->unit_cnt, db->sort, db->unit_link, gu,
                                   p.group_min_writes, st));
        launches += gcc::occ_form_units_launches(db->d.n_records);
    }
    const int block = (int)p.warps_per_block * 32;
    const uint32_t slots = block / p.lanes_per_txn;
    const size_t smem = gu >= 2 ? (size_t)slots * gcc::occ_group_stage_bytes(gu, db->d.max_ops_per_txn)
                                : (size_t)slots * db->d.max_ops_per_txn * gcc::STAGE_BYTES_PER_OP;
    const int occ = gu >= 2 ? gcc::kv_occ_group_occupancy(db->d.field_bytes, block, smem)
                    : kv    ? gcc::kv_exec_occupancy(scheme, db->d.field_bytes, block, smem)
                            : gcc::oe_exec_occupancy(scheme, block, smem);
    if (occ <= 0)
        return fail(GCC_ERR_INVALID, "launch shape does not fit an SM (%d threads, %zu B shared)",
                    block, smem);
    int per_sm = p.blocks_per_sm ? std::min<int>(p.blocks_per_sm, occ) : occ;
    int64_t grid = (int64_t)db->sm_count * per_sm;
    const int64_t needed = ((int64_t)n_txns + slots - 1) / slots;
    grid = std::max<int64_t>(1, std::min(grid, needed));
    GCC_CK(cudaEventRecord(rec.ev[1], st));
    if (n_txns && a.rq)
        GCC_CK(cudaMemsetAsync(db->rq, 0, (size_t)gcc::RETRY_QUEUES * 8, st));

    if (n_txns) {
        if (gu >= 2)
            GCC_CK(gcc::launch_kv_occ_group(db->d.field_bytes, a, (int)grid, block, smem, st));
        else
            GCC_CK(kv ? gcc::launch_kv_exec(scheme, db->d.field_bytes, a, (int)grid, block, smem, st)
                      : gcc::launch_oe_exec(scheme, a, (int)grid, block, smem, st));
        launches += 1;
    }
    GCC_CK(cudaEventRecord(rec.ev[2], st));
    if (n_txns && scheme == GCC_MVCC) {
        GCC_CK(gcc::launch_mv_flatten(a, db->d.field_bytes, st));
        launches += 1;                                       // flatten (+ a memset)
    }
    if (n_txns && (scheme == GCC_OCC || scheme == GCC_TO || scheme == GCC_MVCC)) {
        GCC_CK(gcc::densify_commit_order(a, db->sort, st));
        launches += 1 + 3 * 4 + 1;                           // emit, 4 sort passes, rank
    }
    if (n_txns && scheme == GCC_DET) {
        GCC_CK(gcc::densify_in_id_order(a, db->fold_flags, db->scan_tmp, st));
        launches += 1 + 3 + 1;                               // flags, scan, ranks
    }
    if (n_txns && scheme == GCC_TICTOC) {
        GCC_CK(gcc::densify_tictoc(a, db->sort, st));
        launches += 3 * (1 + 3 * 4) + 1;                     // 3 x (emit, 4 passes), rank
    }
    GCC_CK(cudaEventRecord(rec.ev[3], st));
    rec.stream = st;
    rec.scheme = scheme;
    rec.n_txns = n_txns;
    rec.launches = launches;
    rec.grid = n_txns ? (uint32_t)grid : 0u;
    rec.used = true;
    db->n_stages++;
    switch (scheme) {
        case GCC_NO_WAIT_2PL:
        case GCC_2PL_WAIT_DIE: db->meta_state = META_ZERO; break;
        case GCC_OCC: db->meta_state = META_OCC; break;
        case GCC_TO: db->meta_state = META_TO; break;
        case GCC_DET: db->meta_state = META_DET; break;
        case GCC_TICTOC: db->meta_state = META_TICTOC; break;
        case GCC_MVCC: db->meta_state = n_txns ? META_ZERO : db->meta_state; break;
    }
    db->last_stream = st;
    db->last_scheme = scheme;
    db->last_n_txns = n_txns;
    return GCC_OK;
}

// Stage times of a completed execution (its events must have been reached).
gcc_stage_times stage_times(const StageRec& r) {
    gcc_stage_times t{};
    float a = 0.f, b = 0.f, c = 0.f;
    if (cudaEventElapsedTime(&a, r.ev[0], r.ev[1]) == cudaSuccess) t.prep_ms = a;
    if (cudaEventElapsedTime(&b, r.ev[1], r.ev[2]) == cudaSuccess) t.kernel_ms = b;
    if (cudaEventElapsedTime(&c, r.ev[2], r.ev[3]) == cudaSuccess) t.order_ms = c;
    t.scheme = r.scheme;
    t.n_txns = r.n_txns;
    t.kernel_launches = r.launches;
    t.grid_blocks = r.grid;
    return t;
}

void fill_stats(const gcc::BatchState& h, gcc_scheme scheme, uint64_t n_txns,
                const StageRec* r, gcc_batch_stats* s) {
    *s = gcc_batch_stats{};
    s->n_txns = n_txns;
    s->committed = h.committed;
    s->aborts = h.aborts;
    s->timeouts = h.timeouts;
    s->invalid = h.invalid;
    s->max_attempts = h.max_attempts;
    s->atomics = h.atomics;
    s->device_error = h.error;
    s->scheme = scheme;
    if (r && r->used) {
        const gcc_stage_times t = stage_times(*r);
        s->prep_ms = t.prep_ms;
        s->kernel_ms = t.kernel_ms;
        s->order_ms = t.order_ms;
        s->kernel_launches = t.kernel_launches;
        s->grid_blocks = t.grid_blocks;
    }
}

}  // namespace rt
}  // namespace gcc

using namespace gcc::rt;

namespace gcc {
gcc_status set_error(gcc_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace gcc

extern "C" {

const char* gcc_last_error(void) { return g_err.c_str(); }

gcc_status gcc_default_params(gcc_exec_params* p) {
    if (!p) return fail(GCC_ERR_INVALID, "null params");
    *p = defaults();
    return GCC_OK;
}

gcc_status gcc_db_create(const gcc_db_desc* desc, gcc_db** out) { return create_impl(desc, out); }

gcc_status gcc_db_destroy(gcc_db* db) {
    if (db) free_db(db);
    return GCC_OK;
}

uint32_t gcc_table_count(const gcc_db* db) {
    if (!db) return 0;
    return db->d.schema == GCC_SCHEMA_KV ? 1u : (uint32_t)OE_NCOLS;
}

uint64_t gcc_table_bytes(const gcc_db* db, uint32_t id) {
    if (!db) return 0;
    if (db->d.schema == GCC_SCHEMA_KV) return id == 0 ? db->table_bytes : 0;
    return id < (uint32_t)OE_NCOLS ? db->col_bytes[id] : 0;
}

static void* table_ptr(gcc_db* db, uint32_t id) {
    return db->d.schema == GCC_SCHEMA_KV ? (void*)db->table : (void*)db->cols[id];
}

gcc_status gcc_load_table(gcc_db* db, uint32_t id, const void* src, uint64_t nbytes,
                          int src_on_device) {
    if (!db || !src) return fail(GCC_ERR_INVALID, "null argument");
    const uint64_t want = gcc_table_bytes(db, id);
    if (want == 0) return fail(GCC_ERR_INVALID, "no table %u", id);
    if (nbytes != want)
        return fail(GCC_ERR_INVALID, "table %u holds %llu bytes, got %llu", id,
                    (unsigned long long)want, (unsigned long long)nbytes);
    GCC_CK(cudaSetDevice(db->d.device));
    GCC_CK(cudaDeviceSynchronize());
    GCC_CK(cudaMemcpy(table_ptr(db, id), src, nbytes,
                      src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    GCC_CK(cudaMemset(db->meta, 0, db->n_meta * 16));
    db->meta_state = META_ZERO;
    if (db->d.schema == GCC_SCHEMA_ORDER_ENTRY &&
        (id == (uint32_t)gcc::rt::OE_C_LAST || id == (uint32_t)gcc::rt::OE_C_FIRST))
        GCC_CK(gcc::build_name_index(db->cols[gcc::rt::OE_C_LAST], db->cols[gcc::rt::OE_C_FIRST],
                                     db->d.n_warehouses * gcc::rt::OE_DIST, db->name_idx,
                                     db->name_last, nullptr));
    GCC_CK(cudaDeviceSynchronize());
    return GCC_OK;
}

gcc_status gcc_init_table_seeded(gcc_db* db, uint32_t id, uint64_t seed) {
    if (!db) return fail(GCC_ERR_INVALID, "null database");
    if (db->d.schema != GCC_SCHEMA_KV)
        return fail(GCC_ERR_INVALID,
                    "seeded initialisation is for key-value tables (order-entry tables load "
                    "with gcc_load_table)");
    if (id != 0) return fail(GCC_ERR_INVALID, "no table %u", id);
    GCC_CK(cudaSetDevice(db->d.device));
    GCC_CK(cudaDeviceSynchronize());
    GCC_CK(gcc::launch_seeded_init(db->table, db->d.n_records, db->d.n_fields, db->d.field_bytes,
                                   seed, db->sm_count, 0));
    GCC_CK(cudaMemset(db->meta, 0, db->n_meta * 16));
    db->meta_state = META_ZERO;
    GCC_CK(cudaDeviceSynchronize());
    return GCC_OK;
}

gcc_status gcc_db_read_table(gcc_db* db, uint32_t id, void* dst, uint64_t nbytes,
                             int dst_on_device) {
    if (!db || !dst) return fail(GCC_ERR_INVALID, "null argument");
    const uint64_t want = gcc_table_bytes(db, id);
    if (want == 0) return fail(GCC_ERR_INVALID, "no table %u", id);
    if (nbytes != want)
        return fail(GCC_ERR_INVALID, "table %u holds %llu bytes, got %llu", id,
                    (unsigned long long)want, (unsigned long long)nbytes);
    GCC_CK(cudaSetDevice(db->d.device));
    GCC_CK(cudaDeviceSynchronize());
    GCC_CK(cudaMemcpy(dst, table_ptr(db, id), nbytes,
                      dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return GCC_OK;
}

gcc_status gcc_execute(gcc_db* db, gcc_scheme scheme, const gcc_txn* d_txns, uint32_t n_txns,
                       const gcc_op* d_ops, const gcc_operand* d_operands, uint64_t n_ops,
                       const gcc_exec_params* params, gcc_txn_result* d_results,
                       gcc_operand* d_reads, void* stream) {
    return execute_impl(db, scheme, d_txns, n_txns, d_ops, d_operands, n_ops, params, d_results,
                        d_reads, static_cast<cudaStream_t>(stream));
}

gcc_status gcc_last_stats(gcc_db* db, gcc_batch_stats* stats) {
    if (!db || !stats) return fail(GCC_ERR_INVALID, "null argument");
    GCC_CK(cudaSetDevice(db->d.device));
    gcc::BatchState h{};
    GCC_CK(cudaStreamSynchronize(db->last_stream ? db->last_stream : db->stream));
    GCC_CK(cudaMemcpy(&h, db->st, sizeof h, cudaMemcpyDeviceToHost));
    const StageRec* r = db->n_stages ? &db->stages[(db->n_stages - 1) % STAGE_RING] : nullptr;
    fill_stats(h, db->last_scheme, db->last_n_txns, r, stats);
    return GCC_OK;
}

gcc_status gcc_stage_history(gcc_db* db, uint32_t max_entries, gcc_stage_times* out,
                             uint32_t* n_out) {
    if (!db || !n_out || (max_entries && !out)) return fail(GCC_ERR_INVALID, "null argument");
    GCC_CK(cudaSetDevice(db->d.device));
    const uint64_t avail = std::min<uint64_t>(db->n_stages, STAGE_RING);
    const uint64_t n = std::min<uint64_t>(avail, max_entries);
    for (uint64_t i = 0; i < n; ++i) {
        const StageRec& r = db->stages[(db->n_stages - n + i) % STAGE_RING];
        GCC_CK(cudaEventSynchronize(r.ev[3]));
        out[i] = stage_times(r);
    }
    *n_out = (uint32_t)n;
    return GCC_OK;
}

gcc_status gcc_txn_batch_submit(gcc_db* db, gcc_scheme scheme, const gcc_txn* txns,
                                uint32_t n_txns, const gcc_op* ops, const gcc_operand* operands,
                                uint64_t n_ops, int inputs_on_device,
                                const gcc_exec_params* params, void* stream, gcc_batch** out) {
    if (!db || !out) return fail(GCC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (n_txns > db->d.max_batch_txns || n_ops > db->d.max_batch_ops)
        return fail(GCC_ERR_CAPACITY, "batch exceeds the database maxima");
    if (db->free_h_states.empty())
        return fail(GCC_ERR_CAPACITY, "%u batches outstanding on this database (free some first)",
                    db->n_h_states);
    GCC_CK(cudaSetDevice(db->d.device));
    gcc_batch* b = new (std::nothrow) gcc_batch();
    if (!b) return fail(GCC_ERR_NOMEM, "host allocation failed");
    b->db = db;
    b->stream = stream ? static_cast<cudaStream_t>(stream) : db->stream;
    b->scheme = scheme;
    b->n_txns = n_txns;
    b->n_ops = n_ops;
    b->h_slot = db->free_h_states.back();
    db->free_h_states.pop_back();
    b->h_state = &db->h_states[b->h_slot];
    auto bail = [&](gcc_status s) {
        gcc_batch_free(b);
        return s;
    };
    if (cudaEventCreate(&b->ev_start) != cudaSuccess || cudaEventCreate(&b->ev_done) != cudaSuccess)
        return bail(fail(GCC_ERR_CUDA, "cannot create events"));
    const uint64_t tb = (uint64_t)n_txns * sizeof(gcc_txn), ob = n_ops * sizeof(gcc_op),
                   pb = n_ops * sizeof(gcc_operand);
    const gcc_txn* d_txns = txns;
    const gcc_op* d_ops = ops;
    const gcc_operand* d_operands = operands;
    cudaError_t e;
    if (!inputs_on_device && (tb + ob + pb) > 0) {
        const uint64_t pad = 256;
        e = cudaMallocAsync(&b->d_in, tb + ob + pb + 3 * pad, b->stream);
        if (e != cudaSuccess) return bail(fail(GCC_ERR_NOMEM, "input staging: %s", cudaGetErrorString(e)));
        char* base = static_cast<char*>(b->d_in);
        char* pt = base;
        char* po = base + ((tb + pad - 1) / pad) * pad;
        char* pp = po + ((ob + pad - 1) / pad) * pad;
        if ((tb && cudaMemcpyAsync(pt, txns, tb, cudaMemcpyHostToDevice, b->stream)) ||
            (ob && cudaMemcpyAsync(po, ops, ob, cudaMemcpyHostToDevice, b->stream)) ||
            (pb && cudaMemcpyAsync(pp, operands, pb, cudaMemcpyHostToDevice, b->stream)))
            return bail(fail(GCC_ERR_CUDA, "input upload failed"));
        d_txns = reinterpret_cast<const gcc_txn*>(pt);
        d_ops = reinterpret_cast<const gcc_op*>(po);
        d_operands = reinterpret_cast<const gcc_operand*>(pp);
    }
    if (n_txns && cudaMallocAsync(&b->d_results, (uint64_t)n_txns * sizeof(gcc_txn_result), b->stream))
        return bail(fail(GCC_ERR_NOMEM, "result buffer"));
    if (n_ops && cudaMallocAsync(&b->d_reads, n_ops * sizeof(gcc_operand), b->stream))
        return bail(fail(GCC_ERR_NOMEM, "read-value buffer"));
    if (cudaEventRecord(b->ev_start, b->stream)) return bail(fail(GCC_ERR_CUDA, "event record"));
    b->stage_index = db->n_stages;
    gcc_status s = execute_impl(db, scheme, d_txns, n_txns, d_ops, d_operands, n_ops, params,
                                b->d_results, b->d_reads, b->stream);
    if (s) return bail(s);
    if (cudaMemcpyAsync(b->h_state, db->st, sizeof(gcc::BatchState), cudaMemcpyDeviceToHost,
                        b->stream) ||
        cudaEventRecord(b->ev_done, b->stream))
        return bail(fail(GCC_ERR_CUDA, "batch completion record"));
    *out = b;
    return GCC_OK;
}

gcc_status gcc_batch_wait(gcc_batch* b, uint64_t timeout_ns, gcc_txn_result* results,
                          gcc_operand* read_values, gcc_batch_stats* stats, int outputs_on_device) {
    if (!b) return fail(GCC_ERR_INVALID, "null batch");
    GCC_CK(cudaSetDevice(b->db->d.device));
    const auto t0 = std::chrono::steady_clock::now();
    for (uint32_t spin = 0;; ++spin) {
        cudaError_t q = cudaEventQuery(b->ev_done);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return fail(GCC_ERR_CUDA, "batch failed: %s", cudaGetErrorString(q));
        const uint64_t waited = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                    std::chrono::steady_clock::now() - t0).count();
        if (timeout_ns != UINT64_MAX && waited >= timeout_ns)
            return fail(GCC_ERR_TIMEOUT, "batch still running after %llu ns",
                        (unsigned long long)waited);
        if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    const cudaMemcpyKind k = outputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (results && b->n_txns)
        GCC_CK(cudaMemcpyAsync(results, b->d_results, (uint64_t)b->n_txns * sizeof(gcc_txn_result), k,
                               b->stream));
    if (read_values && b->n_ops)
        GCC_CK(cudaMemcpyAsync(read_values, b->d_reads, b->n_ops * sizeof(gcc_operand), k, b->stream));
    GCC_CK(cudaStreamSynchronize(b->stream));
    gcc::BatchState h = *b->h_state;
    if (stats) {
        const gcc_db* db = b->db;
        const bool live = db->n_stages - b->stage_index <= STAGE_RING;
        fill_stats(h, b->scheme, b->n_txns,
                   live ? &db->stages[b->stage_index % STAGE_RING] : nullptr, stats);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev_start, b->ev_done) == cudaSuccess) stats->elapsed_ms = ms;
    }
    if (h.error) return fail(GCC_ERR_DEVICE, "device reported error flags 0x%x", h.error);
    return GCC_OK;
}

gcc_status gcc_batch_free(gcc_batch* b) {
    if (!b) return GCC_OK;
    cudaSetDevice(b->db->d.device);
    if (b->ev_done) cudaEventSynchronize(b->ev_done);
    else cudaStreamSynchronize(b->stream);
    if (b->d_in) cudaFreeAsync(b->d_in, b->stream);
    if (b->d_results) cudaFreeAsync(b->d_results, b->stream);
    if (b->d_reads) cudaFreeAsync(b->d_reads, b->stream);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->h_slot != UINT32_MAX) b->db->free_h_states.push_back(b->h_slot);
    delete b;
    return GCC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
namespace {

// Committed transactions per second of `reps` executions with params p.
gcc_status measure_point(gcc_db* db, gcc_scheme scheme, const gcc_txn* t, uint32_t n_txns,
                         const gcc_op* o, const gcc_operand* od, uint64_t n_ops,
                         gcc_txn_result* r, gcc_operand* rd, const gcc_exec_params& p,
                         uint32_t warmup, uint32_t reps, cudaStream_t st, double* rate) {
    *rate = 0.0;
    for (uint32_t i = 0; i < warmup; ++i) {
        gcc_status s = execute_impl(db, scheme, t, n_txns, o, od, n_ops, &p, r, rd, st);
        if (s) return s;
    }
    cudaEvent_t e0, e1;
    GCC_CK(cudaEventCreate(&e0));
    GCC_CK(cudaEventCreate(&e1));
    uint64_t committed = 0;
    gcc_status s = GCC_OK;
    float ms = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess) s = fail(GCC_ERR_CUDA, "event record");
    for (uint32_t i = 0; !s && i < reps; ++i) {
        s = execute_impl(db, scheme, t, n_txns, o, od, n_ops, &p, r, rd, st);
        if (!s) {
            // each execution resets the batch state, so read it before the next
            gcc::BatchState h{};
            if (cudaMemcpyAsync(&h, db->st, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                s = fail(GCC_ERR_CUDA, "batch state read");
            committed += h.committed;
        }
    }
    if (!s && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        s = fail(GCC_ERR_CUDA, "event timing");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!s && ms > 0.f) *rate = (double)committed / (ms * 1e-3);
    return s;
}

}  // namespace

extern "C" gcc_status gcc_autotune(gcc_db* db, gcc_scheme scheme, const gcc_txn* d_txns,
                                   uint32_t n_txns, const gcc_op* d_ops,
                                   const gcc_operand* d_operands, uint64_t n_ops,
                                   gcc_txn_result* d_results, gcc_operand* d_reads,
                                   const gcc_tune_space* space, gcc_exec_params* best,
                                   gcc_tune_report* report, void* stream) {
    if (!db || !best) return fail(GCC_ERR_INVALID, "null argument");
    GCC_CK(cudaSetDevice(db->d.device));
    gcc_tune_space sp{};
    if (space) sp = *space;
    static const uint32_t def_lanes[] = {2, 4, 8, 16, 32};
    static const uint32_t def_warps[] = {4, 8, 16, 32};
    static const uint32_t def_caps[] = {65536u, 1000000u, 16000000u};
    if (!sp.n_lanes) { sp.n_lanes = 5; std::memcpy(sp.lanes, def_lanes, sizeof def_lanes); }
    if (!sp.n_warps) { sp.n_warps = 4; std::memcpy(sp.warps, def_warps, sizeof def_warps); }
    if (!sp.n_caps) { sp.n_caps = 3; std::memcpy(sp.caps, def_caps, sizeof def_caps); }
    if (sp.n_lanes > 6 || sp.n_warps > 8 || sp.n_caps > 4)
        return fail(GCC_ERR_INVALID, "tune space lists are too long");
    const uint32_t steps = sp.steps ? sp.steps : 2;
    const uint32_t warmup = sp.warmup ? sp.warmup : 1;
    const uint64_t deadline = sp.point_deadline_ns ? sp.point_deadline_ns : 5000000000ull;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : db->stream;

    gcc_tune_report rep{};
    gcc_exec_params dflt = defaults();
    dflt.deadline_ns = deadline;
    gcc_status s = measure_point(db, scheme, d_txns, n_txns, d_ops, d_operands, n_ops, d_results,
                                 d_reads, dflt, warmup, steps, st, &rep.default_txn_per_s);
    if (s) return s;
    gcc_exec_params winner = dflt;
    double best_rate = rep.default_txn_per_s;
    for (uint32_t li = 0; li < sp.n_lanes; ++li)
        for (uint32_t wi = 0; wi < sp.n_warps; ++wi)
            for (uint32_t ci = 0; ci < sp.n_caps; ++ci) {
                gcc_exec_params p = dflt;
                p.lanes_per_txn = sp.lanes[li];
                p.warps_per_block = sp.warps[wi];
                p.backoff_cap_ns = sp.caps[ci];
                if (validate_params(p)) { g_err.clear(); continue; }
                const int block = (int)p.warps_per_block * 32;
                const size_t smem = (size_t)(block / p.lanes_per_txn) * db->d.max_ops_per_txn *
                                    gcc::STAGE_BYTES_PER_OP;
                const bool kv = db->d.schema == GCC_SCHEMA_KV;
                const int occ = kv ? gcc::kv_exec_occupancy(scheme, db->d.field_bytes, block, smem)
                                   : gcc::oe_exec_occupancy(scheme, block, smem);
                if (occ <= 0) continue;                          // shape does not fit
                double rate = 0.0;
                s = measure_point(db, scheme, d_txns, n_txns, d_ops, d_operands, n_ops, d_results,
                                  d_reads, p, warmup, steps, st, &rate);
                if (s) return s;
                if (rate > best_rate) {
                    best_rate = rate;
                    winner = p;
                    rep.best_index = rep.points;
                }
                rep.points++;
            }
    winner.deadline_ns = defaults().deadline_ns;
    *best = winner;
    rep.best_txn_per_s = best_rate;
    if (report) *report = rep;
    return GCC_OK;
}
