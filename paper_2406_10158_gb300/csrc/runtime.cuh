// runtime.cuh -- host-side objects of the engine shared by the C-ABI
// translation units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <vector>

#include "engine.cuh"

namespace gcc {
namespace rt {

constexpr int OE_NCOLS = 24;
constexpr int OE_C_LAST = 22, OE_C_FIRST = 23;
constexpr uint32_t OE_ITEMS = 100000, OE_DIST = 10, OE_CUST = 3000, OE_LINES = 15;

// Rows of each order-entry column, in table-id order.
inline uint64_t oe_rows(uint32_t col, uint64_t W, uint64_t cap) {
    const uint64_t nd = W * OE_DIST;
    if (col < 2) return W;                          // w_ytd, w_tax
    if (col < 5) return nd;                         // d_ytd, d_tax, d_next_o_id
    if (col < 9) return nd * OE_CUST;               // c_*
    if (col < 10) return OE_ITEMS;                  // i_price
    if (col < 14) return W * OE_ITEMS;              // s_*
    if (col < 18) return nd * cap;                  // o_*, no_flag
    if (col < 22) return nd * cap * OE_LINES;       // ol_*
    return nd * OE_CUST;                            // c_last, c_first
}

enum MetaState { META_ZERO, META_OCC, META_TO, META_DET, META_TICTOC, META_UNKNOWN };

// CUDA events bracketing the stages of one execution.
struct StageRec {
    cudaEvent_t ev[4] = {};        // start, before execute kernel, after it, end
    cudaStream_t stream = nullptr;
    uint32_t scheme = 0, n_txns = 0, launches = 0, grid = 0;
    bool used = false;
};
constexpr uint32_t STAGE_RING = 256;


// Library-internal helpers implemented in api.cu.
gcc_exec_params defaults();
gcc_exec_params merged(const gcc_exec_params* in);
// Aborts before a transaction of `scheme` uses the retry queues.
uint32_t queue_after_for(const gcc_exec_params& p, gcc_scheme scheme);
gcc_status validate_params(const gcc_exec_params& p);
gcc_status fail(gcc_status st, const char* fmt, ...);
// Reset the control words if `scheme` cannot start from their current state.
gcc_status prepare_meta(gcc_db* db, gcc_scheme scheme, cudaStream_t st);
int bit_length(uint64_t v);

}  // namespace rt
}  // namespace gcc

using gcc::rt::MetaState;
using gcc::rt::StageRec;
using gcc::rt::STAGE_RING;
using gcc::rt::META_ZERO;
using gcc::rt::META_OCC;
using gcc::rt::META_TO;
using gcc::rt::META_DET;
using gcc::rt::META_TICTOC;
using gcc::rt::META_UNKNOWN;

struct gcc_db {
    gcc_db_desc d{};
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    // key-value
    uint8_t* table = nullptr;
    uint64_t table_bytes = 0;
    // order-entry
    int64_t* cols[gcc::rt::OE_NCOLS] = {};
    uint64_t col_bytes[gcc::rt::OE_NCOLS] = {};
    int64_t** d_cols = nullptr;
    // concurrency control
    uint64_t* meta = nullptr;
    uint64_t n_meta = 0;
    gcc::BatchState* st = nullptr;
    gcc::DbState* dbs = nullptr;
    uint64_t* rq = nullptr;             // retry queues (gcc::RETRY_QUEUES words)
    MetaState meta_state = META_ZERO;
    // scratch
    gcc::SortScratch sort{};
    uint32_t* scan_tmp = nullptr;
    uint32_t* need = nullptr;
    unsigned long long* order_key = nullptr;
    uint32_t* fold_flags = nullptr;     // deterministic fold: 2 words per transaction
    void* fold_seg = nullptr;           // deterministic fold: tile carries; MVCC values
    uint32_t* mv_slot = nullptr;        // MVCC: version pointer per key-value slot
    uint32_t* unit_cnt = nullptr;       // OCC group commit: writes per record in the batch
    uint32_t* unit_link = nullptr;      // OCC group commit: link word per transaction
    // order-entry: customers by (last, first, number) per district, and the
    // batch's ops with by-name payments resolved
    uint32_t* name_idx = nullptr;
    int64_t* name_last = nullptr;
    uint64_t* ops_resolved = nullptr;
    // latest execution
    cudaStream_t last_stream = nullptr;
    gcc_scheme last_scheme = GCC_OCC;
    uint64_t last_n_txns = 0;
    // pinned copies of BatchState, one per outstanding batch (submitted, not
    // yet freed); free_h_states lists the unused ones
    gcc::BatchState* h_states = nullptr;
    uint32_t n_h_states = 0;
    std::vector<uint32_t> free_h_states;
    // stage timing ring
    StageRec stages[STAGE_RING];
    uint64_t n_stages = 0;
};

struct gcc_batch {
    gcc_db* db = nullptr;
    cudaStream_t stream = nullptr;
    gcc_scheme scheme = GCC_OCC;
    uint32_t n_txns = 0;
    uint64_t n_ops = 0;
    void* d_in = nullptr;                 // staged inputs (host-input batches)
    gcc_txn_result* d_results = nullptr;
    gcc_operand* d_reads = nullptr;
    gcc::BatchState* h_state = nullptr;   // pinned, filled at batch end
    uint32_t h_slot = UINT32_MAX;         // its index in the database's h_states
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    uint64_t stage_index = 0;             // its entry in the database's stage ring
};
