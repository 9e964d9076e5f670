// det_oe.cu -- the deterministic scheme on order-entry batches: every
// record's chain of accesses evaluated in one pass over the sorted access
// table.
//
// The deterministic scheme's outcome is serial execution in transaction-id
// order (Sec. II-C, GPUTx).  That outcome decomposes by record: every
// order-entry op computes its record's new columns from that record's old
// columns and its own operand only, so a record's accesses applied in id order
// from its initial state give exactly the values the serial run reads and the
// record it leaves.  The batch's accesses are sorted by (record, position);
// a warp takes one record segment at a time, holds the record's columns in
// registers and applies the segment's ops in order -- a link of the chain
// costs a few register operations instead of a hand-off through L2.  The
// NewOrder inserts then follow from the values read.
#include <algorithm>

#include "oe_work.cuh"

namespace gcc {
namespace {

using namespace oe;

constexpr int DO_WARPS = 8;                 // warps per block in every kernel here

inline unsigned blocks_for(uint64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// The record classes and their columns, in the register slots c[0..3].
enum Class { WAREHOUSE, DISTRICT, CUSTOMER, STOCK };
__constant__ int CLASS_COLS[4][4] = {
    {W_YTD, W_TAX, -1, -1},
    {D_YTD, D_TAX, D_NEXT_O_ID, -1},
    {C_BALANCE, C_YTD_PAYMENT, C_PAYMENT_CNT, C_DISCOUNT},
    {S_QUANTITY, S_YTD, S_ORDER_CNT, S_REMOTE_CNT},
};

__device__ __forceinline__ int class_of(uint32_t kind) {
    switch (kind) {
        case GCC_OE_W_READ:
        case GCC_OE_W_PAY: return WAREHOUSE;
        case GCC_OE_D_NEWORDER:
        case GCC_OE_D_PAY: return DISTRICT;
        case GCC_OE_C_READ:
        case GCC_OE_C_PAY: return CUSTOMER;
        default: return STOCK;
    }
}

struct Record {
    uint64_t c[4];
};

// One op on the record held in registers: returns the value the op reads and
// updates the record (the same arithmetic as the execute kernel's policy).
__device__ __forceinline__ ulonglong2 apply(Record& r, uint64_t d, ulonglong2 opd) {
    const uint64_t h = opd.x;
    switch (op_kind(d)) {
        case GCC_OE_W_READ: return make_ulonglong2(r.c[1], 0ull);
        case GCC_OE_W_PAY: {
            const ulonglong2 v = make_ulonglong2(r.c[0], 0ull);
            r.c[0] += h;
            return v;
        }
        case GCC_OE_D_NEWORDER: {
            const ulonglong2 v = make_ulonglong2(r.c[2], r.c[1]);
            r.c[2] += 1;
            return v;
        }
        case GCC_OE_D_PAY: {
            const ulonglong2 v = make_ulonglong2(r.c[0], 0ull);
            r.c[0] += h;
            return v;
        }
        case GCC_OE_C_READ: return make_ulonglong2(r.c[3], r.c[0]);
        case GCC_OE_C_PAY: {
            const ulonglong2 v = make_ulonglong2(r.c[0], r.c[2]);
            r.c[0] -= h;
            r.c[1] += h;
            r.c[2] += 1;
            return v;
        }
        default: {                                   // S_NEWORDER
            const ulonglong2 v = make_ulonglong2(r.c[0], r.c[2]);
            const int64_t q = (int64_t)r.c[0], qty = (int64_t)opd.x;
            r.c[0] = (uint64_t)(q >= qty + 10 ? q - qty : q - qty + 91);
            r.c[1] += opd.x;
            r.c[2] += 1;
            r.c[3] += opd.y;
            return v;
        }
    }
}

// Warehouse, district and customer ops only add to their record's columns
// (Payment amounts, the order counter), so a run of them is a prefix sum: the
// value an op reads is the record before the run plus the deltas of the ops
// before it.  delta() gives an op's additions, read_of() what it reads from
// the record as it stands before the op (the values apply() returns).
__device__ __forceinline__ Record delta(uint64_t d, ulonglong2 opd) {
    Record e{};
    const uint64_t h = opd.x;
    switch (op_kind(d)) {
        case GCC_OE_W_PAY:
        case GCC_OE_D_PAY: e.c[0] = h; break;
        case GCC_OE_D_NEWORDER: e.c[2] = 1; break;
        case GCC_OE_C_PAY:
            e.c[0] = 0ull - h;
            e.c[1] = h;
            e.c[2] = 1;
            break;
        default: break;                              // reads
    }
    return e;
}
__device__ __forceinline__ ulonglong2 read_of(uint64_t d, const Record& b) {
    switch (op_kind(d)) {
        case GCC_OE_W_READ: return make_ulonglong2(b.c[1], 0ull);
        case GCC_OE_D_NEWORDER: return make_ulonglong2(b.c[2], b.c[1]);
        case GCC_OE_C_READ: return make_ulonglong2(b.c[3], b.c[0]);
        case GCC_OE_C_PAY: return make_ulonglong2(b.c[0], b.c[2]);
        default: return make_ulonglong2(b.c[0], 0ull);   // W_PAY, D_PAY
    }
}

__global__ void do_fill_none(uint32_t* __restrict__ keys, uint64_t n, uint32_t none) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = none;
}

// Warp per transaction: the checks of the execute kernel, then the access
// entries (record, op position) of a valid transaction's controlled ops; item
// reads (never written) are answered here.  Invalid transactions never run and
// leave no entries.
__global__ void __launch_bounds__(DO_WARPS * 32)
do_validate(const ExecArgs a, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
            uint32_t* __restrict__ valid_flag, uint32_t none) {
    __shared__ uint64_t sdesc[DO_WARPS][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warps = gridDim.x * DO_WARPS;
    unsigned invalid = 0;
    for (uint32_t t = blockIdx.x * DO_WARPS + wib; t < a.n_txns; t += warps) {
        const gcc_txn tx = a.txns[t];
        const uint32_t nops = tx.n_ops;
        const uint64_t first = tx.first_op;
        bool bad = nops > a.max_ops || nops > 64 || !OeWork::valid_txn(a, tx) ||
                   first + nops > a.n_ops;
        if (!bad) {
            for (uint32_t j = lane; j < nops; j += 32) {
                const uint64_t d = a.ops[first + j];
                sdesc[wib][j] = d;
                if (!OeWork::valid_op(a, d)) bad = true;
            }
        }
        __syncwarp();
        bad = __any_sync(0xffffffffu, bad);
        if (!bad) {
            for (uint32_t j = lane; j < nops; j += 32) {
                const uint32_t rj = OeWork::rec(a, sdesc[wib][j]);
                if (rj == NO_CC) continue;
                for (uint32_t i = 0; i < j; ++i)
                    if (OeWork::rec(a, sdesc[wib][i]) == rj) bad = true;
            }
            const Stage S{sdesc[wib], nullptr, nullptr, nullptr, nullptr};
            if (!OeWork::valid_shape(a, S, nops, tx.type)) bad = true;
        }
        bad = __any_sync(0xffffffffu, bad);
        if (first + nops <= a.n_ops) {
            for (uint32_t j = lane; j < nops; j += 32) {
                const uint64_t d = a.ops[first + j];
                const uint32_t r = bad ? NO_CC : OeWork::rec(a, d);
                keys[first + j] = r == NO_CC ? none : r;
                vals[first + j] = (uint32_t)(first + j);
                if (!bad && r == NO_CC) a.reads[first + j] = OeWork::load(a, d);
            }
        }
        if (lane == 0) {
            valid_flag[t] = bad ? 0u : 1u;
            if (bad) a.results[t] = gcc_txn_result{GCC_TXN_INVALID, 0u, ~0ull};
            invalid += bad;
        }
        __syncwarp();
    }
    if (lane == 0 && invalid) {
        atomicAdd(&a.st->invalid, (unsigned long long)invalid);
        atomicOr(&a.st->error, GCC_DEVERR_INVALID);
    }
}

__global__ void do_heads(const uint32_t* __restrict__ sk, uint64_t n, uint32_t* __restrict__ head) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) head[i] = (i == 0 || sk[i] != sk[i - 1]) ? 1u : 0u;
}

// hscan = exclusive count of segment starts: segment s starts at hpos[s].
__global__ void do_head_pos(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ hscan,
                            uint64_t n, uint32_t* __restrict__ hpos) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || sk[i] != sk[i - 1])) hpos[hscan[i]] = (uint32_t)i;
}

// Persistent warps take record segments from a counter (segments differ in
// length by orders of magnitude: a warehouse row is in every transaction of a
// one-warehouse batch).  Per segment: load the record's columns, apply its
// ops 32 at a time -- the warp stages them in shared memory, lane 0 applies
// them in order while the next 32 are loaded, the warp writes the values
// read -- and store the record.
__global__ void __launch_bounds__(DO_WARPS * 32)
do_segments(const ExecArgs a, const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
            const uint32_t* __restrict__ hscan, const uint32_t* __restrict__ hpos, uint64_t n,
            uint32_t none) {
    __shared__ uint64_t s_d[DO_WARPS][32];
    __shared__ ulonglong2 s_o[DO_WARPS][32];
    __shared__ ulonglong2 s_r[DO_WARPS][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t nseg = hscan[n - 1] + ((n == 1 || sk[n - 1] != sk[n - 2]) ? 1u : 0u);
    for (;;) {
        unsigned long long sg = 0;
        if (lane == 0) sg = atomicAdd(&a.st->fetch, 1ull);
        sg = __shfl_sync(0xffffffffu, sg, 0);
        if (sg >= nseg) break;
        const uint64_t start = hpos[sg];
        const uint64_t end = sg + 1 < nseg ? hpos[sg + 1] : n;
        if (sk[start] == none) continue;
        // this lane's op of the first 32
        uint32_t v = 0;
        uint64_t d = 0;
        ulonglong2 o = make_ulonglong2(0ull, 0ull);
        if (start + lane < end) {
            v = sv[start + lane];
            d = a.ops[v];
            o = a.operands[v];
        }
        // the record: its table from the first op's kind, its row from the key
        const uint64_t d0 = __shfl_sync(0xffffffffu, d, 0);
        const int cls = class_of(op_kind(d0));
        const uint32_t row = op_key(d0);
        Record r{};
        if (lane == 0)
            for (int c = 0; c < 4; ++c)
                if (CLASS_COLS[cls][c] >= 0) r.c[c] = OeWork::get(a, CLASS_COLS[cls][c], row);
        // additive classes: every lane holds the record and takes its own op
        if (cls != STOCK)
            for (int c = 0; c < 4; ++c) r.c[c] = __shfl_sync(0xffffffffu, r.c[c], 0);
        for (uint64_t base = start; base < end; base += 32) {
            const uint32_t cnt = (uint32_t)(end - base < 32 ? end - base : 32);
            const uint32_t vcur = v;
            const uint64_t dcur = d;
            const ulonglong2 ocur = o;
            if (cls == STOCK) {
                s_d[wib][lane] = d;
                s_o[wib][lane] = o;
            }
            __syncwarp();
            const uint64_t ni = base + 32 + lane;
            if (ni < end) {
                v = sv[ni];
                d = a.ops[v];
                o = a.operands[v];
            }
            if (cls == STOCK) {
                // the quantity rule is not a sum: lane 0 applies the ops in order
                if (lane == 0)
                    for (uint32_t k = 0; k < cnt; ++k)
                        s_r[wib][k] = apply(r, s_d[wib][k], s_o[wib][k]);
                __syncwarp();
                if ((uint32_t)lane < cnt) a.reads[vcur] = s_r[wib][lane];
                __syncwarp();
            } else {
                // a warp-wide inclusive scan of the column deltas
                const Record e = (uint32_t)lane < cnt ? delta(dcur, ocur) : Record{};
                Record inc = e;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint64_t y = __shfl_up_sync(0xffffffffu, inc.c[c], off);
                        if (lane >= off) inc.c[c] += y;
                    }
                if ((uint32_t)lane < cnt) {
                    Record before = r;
#pragma unroll
                    for (int c = 0; c < 3; ++c) before.c[c] += inc.c[c] - e.c[c];
                    a.reads[vcur] = read_of(dcur, before);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) r.c[c] += __shfl_sync(0xffffffffu, inc.c[c], cnt - 1);
            }
        }
        if (lane == 0)
            for (int c = 0; c < 4; ++c)
                if (CLASS_COLS[cls][c] >= 0) OeWork::put(a, CLASS_COLS[cls][c], row, r.c[c]);
    }
}

// Warp per valid transaction: NewOrder inserts from the values read, and the
// result (commit order = rank among the valid transactions).
__global__ void __launch_bounds__(DO_WARPS * 32)
do_commit(const ExecArgs a, const uint32_t* __restrict__ valid_flag,
          const uint32_t* __restrict__ rank) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warps = gridDim.x * DO_WARPS;
    for (uint32_t t = blockIdx.x * DO_WARPS + wib; t < a.n_txns; t += warps) {
        if (!valid_flag[t]) continue;
        const gcc_txn tx = a.txns[t];
        const uint64_t first = tx.first_op;
        OeWork::insert_new_order(a, (uint32_t)lane, 32u, 0xffffffffu, first, tx.n_ops,
                                 [&](uint32_t j) { return a.ops[first + j]; },
                                 [&](uint32_t j) { return a.reads[first + j]; });
        if (lane == 0) a.results[t] = gcc_txn_result{GCC_TXN_COMMITTED, 1u, rank[t]};
    }
}

__global__ void do_count(const ExecArgs a, const uint32_t* __restrict__ rank,
                         const uint32_t* __restrict__ flag, uint32_t n) {
    if (n) {
        a.st->committed = rank[n - 1] + flag[n - 1];
        a.st->max_attempts = a.st->committed ? 1ull : 0ull;
    }
}

}  // namespace

int det_serial_oe_launches(int key_bits) { return 13 + 3 * ((key_bits + 7) / 8); }

cudaError_t det_serial_oe(const ExecArgs& a, SortScratch& s, uint32_t* scan_tmp, uint32_t* flags,
                          uint32_t* heads, int key_bits, int sm_count, cudaStream_t st) {
    const uint64_t n = a.n_ops;
    const uint32_t none = (uint32_t)a.n_meta;             // sorts after every record
    const unsigned grid_txn = std::min<unsigned>(blocks_for(a.n_txns, DO_WARPS),
                                                 (unsigned)sm_count * 16u);
    if (n) do_fill_none<<<blocks_for(n, 256), 256, 0, st>>>(s.k0, n, none);
    if (a.n_txns) do_validate<<<grid_txn, DO_WARPS * 32, 0, st>>>(a, s.k0, s.v0, flags, none);
    if (n) {
        uint32_t *sk = s.k0, *sv = s.v0;
        cudaError_t e = radix_sort_pairs(s, n, key_bits, &sk, &sv, st);
        if (e != cudaSuccess) return e;
        uint32_t* hpos = sk == s.k0 ? s.k1 : s.k0;        // the buffer the sort left free
        do_heads<<<blocks_for(n, 256), 256, 0, st>>>(sk, n, heads);
        e = exclusive_scan_u32(heads, n, scan_tmp, st);
        if (e != cudaSuccess) return e;
        do_head_pos<<<blocks_for(n, 256), 256, 0, st>>>(sk, heads, n, hpos);
        do_segments<<<(unsigned)sm_count * 4u, DO_WARPS * 32, 0, st>>>(a, sk, sv, heads, hpos, n,
                                                                      none);
    }
    if (a.n_txns) {
        uint32_t* rank = flags + a.n_txns;
        cudaError_t e = cudaMemcpyAsync(rank, flags, (size_t)a.n_txns * 4,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = exclusive_scan_u32(rank, a.n_txns, scan_tmp, st);
        if (e != cudaSuccess) return e;
        do_commit<<<grid_txn, DO_WARPS * 32, 0, st>>>(a, flags, rank);
        do_count<<<1, 1, 0, st>>>(a, rank, flags, a.n_txns);
    }
    return cudaGetLastError();
}

}  // namespace gcc
