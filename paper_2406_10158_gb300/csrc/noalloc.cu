// noalloc.cu -- deterministic execution of a small key-value batch without
// any device allocation by the library.
//
// Some callers cannot allocate device memory: a host application whose
// device memory is reserved up front by another framework's caching
// allocator, or a latency-critical loop in which cudaMalloc's implicit device
// synchronisation is not acceptable.  gcc_det_execute_noalloc serves them:
// the caller passes the table, the batch and the output buffers; all scratch
// (per-record counters, the sorted access table, wait thresholds, batch
// state) lives in one file-scope device array below, which every GPU that
// loads this library holds until the process exits.
#include <mutex>
#include <string>

#include "engine.cuh"

namespace {

constexpr uint32_t NA_MAX = 65536;   // records, ops and transactions per call

// Byte layout of the static scratch (each piece 256-byte aligned).
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t NA_TILES = (NA_MAX + 2047) / 2048;     // radix-sort tiles (of 2048 items or more)
constexpr size_t OFF_META = 0;
constexpr size_t OFF_K0 = OFF_META + align256(NA_MAX * 8);
constexpr size_t OFF_V0 = OFF_K0 + align256(NA_MAX * 4);
constexpr size_t OFF_K1 = OFF_V0 + align256(NA_MAX * 4);
constexpr size_t OFF_V1 = OFF_K1 + align256(NA_MAX * 4);
constexpr size_t OFF_HIST = OFF_V1 + align256(NA_MAX * 4);
constexpr size_t OFF_TOTALS = OFF_HIST + align256(NA_TILES * 256 * 4);
constexpr size_t OFF_SCAN = OFF_TOTALS + align256(256 * 4);
constexpr size_t OFF_NEED = OFF_SCAN + align256(64 * 4);
constexpr size_t OFF_STATE = OFF_NEED + align256(NA_MAX * 4);
constexpr size_t OFF_DBSTATE = OFF_STATE + align256(sizeof(gcc::BatchState));
constexpr size_t NA_BYTES = OFF_DBSTATE + align256(sizeof(gcc::DbState));

__device__ __align__(256) static unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mutex;
constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

gcc_status na_fail(gcc_status s, const std::string& msg) {
    return gcc::set_error(s, msg.c_str());
}

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol itself as a device pointer).
gcc_status scratch_on(int dev, unsigned char** out) {
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(GCC_ERR_INVALID, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return na_fail(GCC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_na_ptr[dev];
    return GCC_OK;
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (maxval) { ++b; maxval >>= 1; }
    return b < 1 ? 1 : b;
}

}  // namespace

extern "C" {

gcc_status gcc_det_execute_noalloc(void* d_table, uint32_t n_records, uint32_t n_fields,
                                   uint32_t field_bytes, const gcc_txn* d_txns, uint32_t n_txns,
                                   const gcc_op* d_ops, const gcc_operand* d_operands,
                                   uint32_t n_ops, uint32_t max_ops_per_txn,
                                   gcc_txn_result* d_results, gcc_operand* d_reads,
                                   void* stream) {
    if (n_records == 0 || n_records > NA_MAX || n_ops > NA_MAX || n_txns > NA_MAX)
        return na_fail(GCC_ERR_CAPACITY,
                       "gcc_det_execute_noalloc handles at most 65536 records, ops and "
                       "transactions per call");
    if (field_bytes != 8 && field_bytes != 16) return na_fail(GCC_ERR_INVALID, "field_bytes must be 8 or 16");
    if (n_fields == 0 || n_fields > 255) return na_fail(GCC_ERR_INVALID, "n_fields must be in 1..255");
    if (max_ops_per_txn == 0 || max_ops_per_txn > 64)
        return na_fail(GCC_ERR_INVALID, "max_ops_per_txn must be in 1..64");
    if (!d_table || (n_txns && (!d_txns || !d_results)) || (n_ops && (!d_ops || !d_operands || !d_reads)))
        return na_fail(GCC_ERR_INVALID, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(GCC_ERR_CUDA, cudaGetErrorString(e));
    unsigned char* base = nullptr;
    gcc_status s = scratch_on(dev, &base);
    if (s) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    gcc::SortScratch sort{};
    sort.k0 = reinterpret_cast<uint32_t*>(base + OFF_K0);
    sort.v0 = reinterpret_cast<uint32_t*>(base + OFF_V0);
    sort.k1 = reinterpret_cast<uint32_t*>(base + OFF_K1);
    sort.v1 = reinterpret_cast<uint32_t*>(base + OFF_V1);
    sort.hist = reinterpret_cast<uint32_t*>(base + OFF_HIST);
    sort.totals = reinterpret_cast<uint32_t*>(base + OFF_TOTALS);
    sort.max_items = NA_MAX;

    gcc::ExecArgs a{};
    a.txns = d_txns;
    a.ops = reinterpret_cast<const uint64_t*>(d_ops);
    a.operands = reinterpret_cast<const ulonglong2*>(d_operands);
    a.n_txns = n_txns;
    a.n_ops = n_ops;
    a.results = d_results;
    a.reads = reinterpret_cast<ulonglong2*>(d_reads);
    a.table = static_cast<uint8_t*>(d_table);
    a.n_records = n_records;
    a.n_fields = n_fields;
    a.meta = reinterpret_cast<uint64_t*>(base + OFF_META);
    a.n_meta = n_records;
    a.need = reinterpret_cast<uint32_t*>(base + OFF_NEED);
    a.st = reinterpret_cast<gcc::BatchState*>(base + OFF_STATE);
    a.dbs = reinterpret_cast<gcc::DbState*>(base + OFF_DBSTATE);
    a.lanes = 16;
    a.max_ops = max_ops_per_txn;
    a.collapse = 1;
    a.max_attempts = 1;
    a.read_retries = 8;
    a.wait_budget_ns = 2000000000ull;
    a.deadline_ns = 60000000000ull;

    // batch state zeroed on every call; record counters are set by the
    // preprocessing for every record the batch touches
    e = gcc::launch_batch_begin(a.st, a.dbs, GCC_DET, st);
    if (e == cudaSuccess && n_ops)
        // the sort covers the key n_records, which marks out-of-range ops, so
        // that they sort after every record's run
        e = gcc::det_prepare(a, sort, reinterpret_cast<uint32_t*>(base + OFF_SCAN),
                             bits_for(n_records), GCC_SCHEMA_KV, st);
    if (e != cudaSuccess) return na_fail(GCC_ERR_CUDA, cudaGetErrorString(e));
    if (n_txns) {
        const int block = 8 * 32;
        const uint32_t slots = block / a.lanes;
        const size_t smem = (size_t)slots * max_ops_per_txn * gcc::STAGE_BYTES_PER_OP;
        const int occ = gcc::kv_exec_occupancy(GCC_DET, field_bytes, block, smem);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return na_fail(GCC_ERR_CUDA, std::string("cannot query the SM count: ") +
                                             cudaGetErrorString(e));
        if (occ <= 0)
            return na_fail(GCC_ERR_INVALID,
                           "launch shape does not fit an SM (" + std::to_string(block) +
                               " threads, " + std::to_string(smem) + " B shared)");
        int64_t grid = (int64_t)sms * occ;
        const int64_t needed = ((int64_t)n_txns + slots - 1) / slots;
        if (grid > needed) grid = needed;
        e = gcc::launch_kv_exec(GCC_DET, field_bytes, a, (int)grid, block, smem, st);
        // dense ranks over the committed transactions; the sort buffers are
        // free again once the wait thresholds exist
        if (e == cudaSuccess)
            e = gcc::densify_in_id_order(a, sort.k1, reinterpret_cast<uint32_t*>(base + OFF_SCAN), st);
        if (e != cudaSuccess) return na_fail(GCC_ERR_CUDA, cudaGetErrorString(e));
    }
    return GCC_OK;
}

}  // extern "C"
