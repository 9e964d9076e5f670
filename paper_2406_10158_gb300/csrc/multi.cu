// multi.cu -- the batched form: many independent key-value batches (each on
// its own database) in one persistent-kernel launch, optionally replayed as a
// CUDA graph.
//
// Lane groups take transactions from one counter over the concatenation of
// all batches, so large and small batches share the GPU without a launch per
// batch; each transaction runs against its own database exactly as in the
// single-batch kernel.  OCC and TO draw timestamps from one clock shared by
// the launch (started above every database's own clock and written back to
// them afterwards), so commit ranks for all batches come from two sorts: by
// timestamp, then stably by batch.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "kv_work.cuh"
#include "runtime.cuh"

namespace gcc {
namespace {

constexpr uint32_t MAX_BATCHES = 256;

struct MultiState {
    unsigned long long fetch;
    unsigned long long total;
    DbState clock;                 // shared OCC / TO clock of the launch
    unsigned long long padded;     // fetch space: chunks rounded up to a power of two
    unsigned int chunk_bits;       // log2 of the number of chunks in it
    unsigned int pad;
};

// Transactions are handed out in chunks of FETCH_CHUNK consecutive ids, the
// chunks in bit-reversed order over the fetch space, so that consecutive
// fetches land far apart -- in different databases -- and every database's
// batch advances at a rate proportional to its size.  Handed out database
// after database instead, the batches' hot-record chains would run one after
// the other, as they do in separate launches.
constexpr uint32_t FETCH_CHUNK_BITS = 5;

__device__ __forceinline__ unsigned long long interleaved_id(unsigned long long g, unsigned bits) {
    const unsigned long long chunk = g >> FETCH_CHUNK_BITS;
    const unsigned long long off = g & ((1ull << FETCH_CHUNK_BITS) - 1);
    const unsigned long long rc = bits ? (__brevll(chunk) >> (64 - bits)) : 0ull;
    return (rc << FETCH_CHUNK_BITS) | off;
}

__device__ __forceinline__ uint32_t find_batch(const uint32_t* prefix, uint32_t n, uint64_t g) {
    uint32_t lo = 0, hi = n;       // prefix[lo] <= g < prefix[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

struct MultiFetch {
    const ExecArgs* args;
    const uint32_t* prefix;        // shared-memory copy, n + 1 entries
    uint32_t n;
    MultiState* ms;
    Counters* c;
    const ExecArgs* cur;

    // Counters of the lane-group leader into the batch they belong to.
    __device__ __forceinline__ void flush(const Lane& L) {
        const uint32_t atoms = __reduce_add_sync(L.gmask, L.n_atom);
        L.n_atom = 0;
        if (cur && L.lig == 0) {
            BatchState* st = cur->st;
            if (atoms) atomicAdd(&st->atomics, (unsigned long long)atoms);
            if (c->commits) atomicAdd(&st->committed, (unsigned long long)c->commits);
            if (c->aborts) atomicAdd(&st->aborts, (unsigned long long)c->aborts);
            if (c->timeouts) atomicAdd(&st->timeouts, (unsigned long long)c->timeouts);
            if (c->invalid) atomicAdd(&st->invalid, (unsigned long long)c->invalid);
            if (c->max_att) atomicMax(&st->max_attempts, (unsigned long long)c->max_att);
        }
        *c = Counters{};
    }
    __device__ __forceinline__ bool next(const Lane& L, uint32_t& t, const ExecArgs*& A) {
        unsigned long long id = 0;
        for (;;) {                 // ids past the last transaction are skipped
            unsigned long long g = 0;
            if (L.lig == 0) g = agg_ticket(&ms->fetch);
            g = __shfl_sync(L.gmask, g, L.gbase);
            if (g >= ms->padded) return false;
            id = interleaved_id(g, ms->chunk_bits);
            if (id < ms->total) break;
        }
        const uint32_t i = find_batch(prefix, n, id);
        A = args + i;
        t = (uint32_t)(id - prefix[i]);
        if (A != cur) {
            flush(L);
            cur = A;
        }
        return true;
    }
    __device__ __forceinline__ void done(const Lane&, const ExecArgs&, Counters&) {}
};

template <int SCHEME, class Work>
__global__ void __launch_bounds__(1024)
multi_kernel(const ExecArgs* __restrict__ args, const uint32_t* __restrict__ prefix, uint32_t n,
             MultiState* ms, uint32_t lanes, uint32_t max_ops, uint64_t deadline_ns) {
    __shared__ uint32_t prefix_s[MAX_BATCHES + 1];
    for (uint32_t i = threadIdx.x; i <= n; i += blockDim.x) prefix_s[i] = prefix[i];
    __syncthreads();
    Lane L;
    Stage S;
    setup_lanes(lanes, max_ops, L, S);
    // one deadline per warp: lanes must agree on every time comparison
    const uint64_t deadline = __shfl_sync(0xffffffffu, globaltimer(), 0) + deadline_ns;
    Counters c;
    MultiFetch F{args, prefix_s, n, ms, &c, nullptr};
    group_loop<SCHEME, Work>(F, L, S, max_ops, deadline, c);
    F.flush(L);
}

// Per-batch states zeroed, the shared clock started above every database's.
__global__ void multi_begin(const ExecArgs* __restrict__ args, DbState* const* __restrict__ own,
                            uint32_t n, MultiState* ms, int scheme) {
    __shared__ unsigned long long occ, to;
    if (threadIdx.x == 0) {
        occ = 0;
        to = 0;
        for (uint32_t i = 0; i < n; ++i) {
            occ = max(occ, own[i]->occ_clock);
            to = max(to, own[i]->to_clock);
        }
        ms->fetch = 0;
        ms->clock.occ_clock = occ;
        ms->clock.to_clock = to;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        BatchState z{};
        // MVCC's timestamps count from 1 in every batch (its own counter)
        z.ticket_base = scheme == GCC_TO ? to : scheme == GCC_MVCC ? 0ull : occ;
        *args[i].st = z;
    }
}

// Zeroes every database's retry queues (grid: queue words x databases).
__global__ void multi_rq_reset(const ExecArgs* __restrict__ args, uint32_t n) {
    const uint32_t i = blockIdx.y;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && args[i].rq && w < RETRY_QUEUES) args[i].rq[w] = 0;
}

// Every database continues its own clock from the shared one.
__global__ void multi_end(DbState* const* __restrict__ own, uint32_t n, const MultiState* ms) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        own[i]->occ_clock = max(own[i]->occ_clock, ms->clock.occ_clock);
        own[i]->to_clock = max(own[i]->to_clock, ms->clock.to_clock);
    }
}

__global__ void multi_rank_keys(const ExecArgs* __restrict__ args, const uint32_t* __restrict__ prefix,
                                uint32_t n, uint64_t total, uint32_t* __restrict__ keys,
                                uint32_t* __restrict__ vals) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const uint32_t i = find_batch(prefix, n, g);
    const ExecArgs& a = args[i];
    const uint32_t t = (uint32_t)(g - prefix[i]);
    uint32_t k = 0xffffffffu;
    if (a.results[t].status == GCC_TXN_COMMITTED) {
        // a 32-bit offset from the plan's starting clock, as in the plain path
        const unsigned long long d = a.order_key[t] - a.st->ticket_base;
        if (d >= 0xffffffffull) atomicOr(&a.st->error, GCC_DEVERR_TS_OVERFLOW);
        k = (uint32_t)d;
    }
    keys[g] = k;
    vals[g] = (uint32_t)g;
}

// After sorting by timestamp: key each position by its batch for a stable
// second sort that groups batches while keeping timestamp order inside.
__global__ void multi_batch_keys(const uint32_t* __restrict__ prefix, uint32_t n, uint64_t total,
                                 uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < total) keys[p] = find_batch(prefix, n, vals[p]);
}

__global__ void multi_ranks(const ExecArgs* __restrict__ args, const uint32_t* __restrict__ prefix,
                            uint32_t n, uint64_t total, const uint32_t* __restrict__ vals) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const uint32_t g = vals[p];
    const uint32_t i = find_batch(prefix, n, g);
    const ExecArgs& a = args[i];
    const uint32_t t = g - prefix[i];
    if (a.results[t].status == GCC_TXN_COMMITTED) a.results[t].commit_order = p - prefix[i];
}

template <int SCHEME, int FB>
int multi_occupancy(int block, size_t smem) {
    return occupancy_of(multi_kernel<SCHEME, KvWork<FB>>, block, smem);
}

template <int SCHEME, int FB>
cudaError_t multi_launch_kernel(const ExecArgs* args, const uint32_t* prefix, uint32_t n,
                                MultiState* ms, uint32_t lanes, uint32_t max_ops,
                                uint64_t deadline_ns, int grid, int block, size_t smem,
                                cudaStream_t st) {
    // the dynamic shared-memory limit was raised when the plan measured occupancy
    multi_kernel<SCHEME, KvWork<FB>><<<grid, block, smem, st>>>(args, prefix, n, ms, lanes, max_ops,
                                                              deadline_ns);
    return cudaGetLastError();
}

int occupancy_for(gcc_scheme scheme, uint32_t fb, int block, size_t smem) {
#define GCC_MULTI_OCC(SC)                                                        \
    case SC:                                                                     \
        return fb == 16 ? multi_occupancy<SC, 16>(block, smem)                   \
                        : multi_occupancy<SC, 8>(block, smem);
    switch (scheme) {
        GCC_MULTI_OCC(GCC_NO_WAIT_2PL)
        GCC_MULTI_OCC(GCC_TO)
        GCC_MULTI_OCC(GCC_OCC)
        GCC_MULTI_OCC(GCC_TICTOC)
        GCC_MULTI_OCC(GCC_2PL_WAIT_DIE)
        GCC_MULTI_OCC(GCC_MVCC)
        default:
            return 0;
    }
#undef GCC_MULTI_OCC
}

// TicToc's serial order over every batch of the plan: three stable passes
// (sequence number, then the timestamp's low and high words; pass 0 keys by
// position, later passes re-key the previous pass's order in place), as in
// the single-batch path; the batch grouping follows.
__global__ void multi_tt_keys(const ExecArgs* __restrict__ args, const uint32_t* __restrict__ prefix,
                              uint32_t n, uint64_t total, int pass, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const uint32_t g = pass == 0 ? (uint32_t)p : vals[p];
    const uint32_t i = find_batch(prefix, n, g);
    const ExecArgs& a = args[i];
    const uint32_t t = g - prefix[i];
    uint32_t k = 0xffffffffu;
    if (a.results[t].status == GCC_TXN_COMMITTED)
        k = pass == 0 ? a.seq[t] : pass == 1 ? (uint32_t)a.order_key[t]
                                             : (uint32_t)(a.order_key[t] >> 32);
    keys[p] = k;
    vals[p] = g;
}

inline unsigned blocks_for(uint64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace
}  // namespace gcc

using namespace gcc::rt;

struct gcc_multi_plan {
    gcc_scheme scheme = GCC_OCC;
    int device = 0;
    uint32_t n = 0;
    uint32_t field_bytes = 8;
    uint64_t total = 0;
    gcc_exec_params p{};
    std::vector<gcc_db*> dbs;
    std::vector<uint32_t> h_prefix;
    gcc::ExecArgs* d_args = nullptr;
    uint32_t* d_prefix = nullptr;
    gcc::DbState** d_own = nullptr;
    gcc::MultiState* d_ms = nullptr;
    gcc::SortScratch sort{};
    int grid = 0, block = 0;
    size_t smem = 0;
    uint32_t max_ops = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    uint32_t launches = 0;
    // deterministic plans: every database's batch by its own prefix-sum
    // pipeline (its own scratch), spread over side streams that fork from and
    // join the launch stream, so that the pipelines overlap
    std::vector<gcc::ExecArgs> h_args;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;     // [0]: fork, [1 + k]: side stream k done
};

namespace {

void free_plan(gcc_multi_plan* pl) {
    cudaSetDevice(pl->device);
    if (pl->stream) cudaStreamSynchronize(pl->stream);
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    cudaFree(pl->d_args);
    cudaFree(pl->d_prefix);
    cudaFree(pl->d_own);
    cudaFree(pl->d_ms);
    cudaFree(pl->sort.k0);
    cudaFree(pl->sort.v0);
    cudaFree(pl->sort.k1);
    cudaFree(pl->sort.v1);
    cudaFree(pl->sort.hist);
    cudaFree(pl->sort.totals);
    for (cudaStream_t s : pl->side)
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    for (cudaEvent_t e : pl->ev)
        if (e) cudaEventDestroy(e);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    delete pl;
}

MetaState state_after(gcc_scheme s) {
    return s == GCC_OCC ? META_OCC : s == GCC_TO ? META_TO : s == GCC_TICTOC ? META_TICTOC
                                                                             : META_ZERO;
}

// Deterministic plans: database i's batch on side stream i mod k, the side
// streams forked from `st` and joined back into it.
gcc_status enqueue_det(gcc_multi_plan* pl, cudaStream_t st) {
    using namespace gcc;
    const uint32_t k = (uint32_t)pl->side.size();
    cudaError_t e = cudaEventRecord(pl->ev[0], st);
    for (uint32_t j = 0; e == cudaSuccess && j < k; ++j) e = cudaStreamWaitEvent(pl->side[j], pl->ev[0], 0);
    uint32_t launches = 0;
    for (uint32_t i = 0; e == cudaSuccess && i < pl->n; ++i) {
        gcc_db* db = pl->dbs[i];
        cudaStream_t s = pl->side[i % k];
        e = launch_batch_begin(db->st, db->dbs, GCC_DET, s);
        if (e == cudaSuccess)
            e = det_fold_kv(pl->h_args[i], pl->field_bytes, db->sort, db->scan_tmp, db->fold_flags,
                            db->fold_seg, s);
        int bits = 0;
        for (uint64_t v = (uint64_t)db->d.n_fields * db->d.n_records; v; v >>= 1) ++bits;
        launches += 1 + 2 + 3 * ((bits + 7) / 8) + 4 + 1 + 3 + 2;
    }
    for (uint32_t j = 0; e == cudaSuccess && j < k; ++j) {
        e = cudaEventRecord(pl->ev[1 + j], pl->side[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, pl->ev[1 + j], 0);
    }
    if (e != cudaSuccess) return fail(GCC_ERR_CUDA, "multi launch: %s", cudaGetErrorString(e));
    pl->launches = launches;
    return GCC_OK;
}

// The launch sequence, all stream-ordered and allocation-free.
gcc_status enqueue(gcc_multi_plan* pl, cudaStream_t st) {
    using namespace gcc;
    if (pl->scheme == GCC_DET) return enqueue_det(pl, st);
    multi_begin<<<1, 256, 0, st>>>(pl->d_args, pl->d_own, pl->n, pl->d_ms, (int)pl->scheme);
    if (pl->n)
        multi_rq_reset<<<dim3(RETRY_QUEUES / 256, pl->n), 256, 0, st>>>(pl->d_args, pl->n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const uint32_t lanes = pl->p.lanes_per_txn;
        const uint64_t dl = pl->p.deadline_ns;
        switch (pl->scheme) {
#define GCC_MULTI_CASE(SC)                                                                         \
    case SC:                                                                                       \
        e = pl->field_bytes == 16                                                                  \
                ? multi_launch_kernel<SC, 16>(pl->d_args, pl->d_prefix, pl->n, pl->d_ms, lanes,     \
                                              pl->max_ops, dl, pl->grid, pl->block, pl->smem, st)  \
                : multi_launch_kernel<SC, 8>(pl->d_args, pl->d_prefix, pl->n, pl->d_ms, lanes,      \
                                             pl->max_ops, dl, pl->grid, pl->block, pl->smem, st);  \
        break;
            GCC_MULTI_CASE(GCC_NO_WAIT_2PL)
            GCC_MULTI_CASE(GCC_TO)
            GCC_MULTI_CASE(GCC_OCC)
            GCC_MULTI_CASE(GCC_TICTOC)
            GCC_MULTI_CASE(GCC_2PL_WAIT_DIE)
            GCC_MULTI_CASE(GCC_MVCC)
#undef GCC_MULTI_CASE
            default:
                e = cudaErrorInvalidValue;
                break;
        }
    }
    uint32_t launches = 3;
    // MVCC: each database's newest versions into its table before the ranks
    // (the version store lives in the database's own scratch)
    for (uint32_t i = 0; e == cudaSuccess && pl->scheme == GCC_MVCC && i < pl->n; ++i) {
        e = launch_mv_flatten(pl->h_args[i], pl->field_bytes, st);
        launches += 1;
    }
    const bool dense = pl->scheme == GCC_NO_WAIT_2PL || pl->scheme == GCC_2PL_WAIT_DIE;
    if (e == cudaSuccess && !dense && pl->total) {
        uint32_t *sk, *sv;
        if (pl->scheme == GCC_TICTOC) {
            // (timestamp, sequence number), by three stable passes
            for (int pass = 0; e == cudaSuccess && pass < 3; ++pass) {
                multi_tt_keys<<<blocks_for(pl->total, 256), 256, 0, st>>>(
                    pl->d_args, pl->d_prefix, pl->n, pl->total, pass, pl->sort.k0, pl->sort.v0);
                e = radix_sort_pairs(pl->sort, pl->total, 32, &sk, &sv, st);
            }
            launches += 3 * (1 + 12);
        } else {
            multi_rank_keys<<<blocks_for(pl->total, 256), 256, 0, st>>>(pl->d_args, pl->d_prefix, pl->n,
                                                                     pl->total, pl->sort.k0, pl->sort.v0);
            e = radix_sort_pairs(pl->sort, pl->total, 32, &sk, &sv, st);   // by timestamp
            launches += 1 + 12;
        }
        if (e == cudaSuccess) {
            multi_batch_keys<<<blocks_for(pl->total, 256), 256, 0, st>>>(pl->d_prefix, pl->n, pl->total,
                                                                      sk, sv);
            // the second sort reads from (k0, v0): four-pass sorts end there
            e = radix_sort_pairs(pl->sort, pl->total, 8, &sk, &sv, st);  // stably by batch
        }
        if (e == cudaSuccess)
            multi_ranks<<<blocks_for(pl->total, 256), 256, 0, st>>>(pl->d_args, pl->d_prefix, pl->n,
                                                                 pl->total, sv);
        launches += 1 + 3 + 1;
    }
    if (e == cudaSuccess) {
        multi_end<<<1, 256, 0, st>>>(pl->d_own, pl->n, pl->d_ms);
        e = cudaGetLastError();
        launches += 1;
    }
    if (e != cudaSuccess) return fail(GCC_ERR_CUDA, "multi launch: %s", cudaGetErrorString(e));
    pl->launches = launches;
    return GCC_OK;
}

}  // namespace

extern "C" {

gcc_status gcc_multi_plan_create(gcc_scheme scheme, const gcc_multi_batch* b, uint32_t n,
                                 const gcc_exec_params* params, gcc_multi_plan** out) {
    if (!b || !out || n == 0) return fail(GCC_ERR_INVALID, "null argument or no batches");
    *out = nullptr;
    if (n > gcc::MAX_BATCHES) return fail(GCC_ERR_CAPACITY, "at most 256 batches per plan");
    if ((unsigned)scheme > GCC_MVCC) return fail(GCC_ERR_INVALID, "unknown scheme %d", (int)scheme);
    gcc_exec_params p = merged(params);
    gcc_status s = validate_params(p);
    if (s) return s;
    const int dev = b[0].db ? b[0].db->d.device : 0;
    uint32_t fb = b[0].db ? b[0].db->d.field_bytes : 8, max_ops = 0;
    uint64_t total = 0;
    std::vector<uint32_t> prefix(n + 1, 0);
    for (uint32_t i = 0; i < n; ++i) {
        gcc_db* db = b[i].db;
        if (!db || db->d.schema != GCC_SCHEMA_KV)
            return fail(GCC_ERR_INVALID, "batch %u: a key-value database is required", i);
        if (db->d.device != dev || db->d.field_bytes != fb)
            return fail(GCC_ERR_INVALID, "batch %u: all databases share one device and slot width", i);
        for (uint32_t j = 0; j < i; ++j)
            if (b[j].db == db) return fail(GCC_ERR_INVALID, "batch %u: database used twice", i);
        if (b[i].n_txns > db->d.max_batch_txns || b[i].n_ops > db->d.max_batch_ops)
            return fail(GCC_ERR_CAPACITY, "batch %u exceeds its database's maxima", i);
        if (scheme == GCC_DET && (uint64_t)db->d.n_fields * db->d.n_records >= (1ull << 32))
            return fail(GCC_ERR_CAPACITY,
                        "batch %u: deterministic batches need n_records * n_fields below 2^32", i);
        if ((b[i].n_txns && (!b[i].d_txns || !b[i].d_results)) ||
            (b[i].n_ops && (!b[i].d_ops || !b[i].d_operands || !b[i].d_reads)))
            return fail(GCC_ERR_INVALID, "batch %u: null pointer", i);
        max_ops = std::max(max_ops, db->d.max_ops_per_txn);
        total += b[i].n_txns;
        prefix[i + 1] = (uint32_t)total;
    }
    if (total >= (1ull << 32)) return fail(GCC_ERR_CAPACITY, "more than 2^32 transactions");
    if (cudaSetDevice(dev) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(GCC_ERR_CUDA, "cannot select device %d", dev);

    gcc_multi_plan* pl = new (std::nothrow) gcc_multi_plan();
    if (!pl) return fail(GCC_ERR_NOMEM, "host allocation failed");
    auto bail = [&](gcc_status st) { free_plan(pl); return st; };
    pl->scheme = scheme;
    pl->device = dev;
    pl->n = n;
    pl->field_bytes = fb;
    pl->total = total;
    pl->p = p;
    pl->h_prefix = prefix;
    pl->max_ops = max_ops;
    if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(GCC_ERR_CUDA, "cannot create stream"));
    auto alloc = [&](void** ptr, size_t bytes) {
        return cudaMalloc(ptr, bytes ? bytes : 1) == cudaSuccess;
    };
    const uint64_t items = std::max<uint64_t>(total, 1);
    if (!alloc((void**)&pl->d_args, sizeof(gcc::ExecArgs) * n) ||
        !alloc((void**)&pl->d_prefix, sizeof(uint32_t) * (n + 1)) ||
        !alloc((void**)&pl->d_own, sizeof(gcc::DbState*) * n) ||
        !alloc((void**)&pl->d_ms, sizeof(gcc::MultiState)) ||
        !alloc((void**)&pl->sort.k0, items * 4) || !alloc((void**)&pl->sort.v0, items * 4) ||
        !alloc((void**)&pl->sort.k1, items * 4) || !alloc((void**)&pl->sort.v1, items * 4) ||
        !alloc((void**)&pl->sort.hist, gcc::sort_max_tiles(items) * 256 * 4) ||
        !alloc((void**)&pl->sort.totals, 256 * 4))
        return bail(fail(GCC_ERR_NOMEM, "cannot allocate the plan"));
    pl->sort.max_items = items;

    std::vector<gcc::ExecArgs> args(n);
    std::vector<gcc::DbState*> own(n);
    for (uint32_t i = 0; i < n; ++i) {
        gcc_db* db = b[i].db;
        pl->dbs.push_back(db);
        own[i] = db->dbs;
        gcc::ExecArgs& a = args[i];
        a = gcc::ExecArgs{};
        a.txns = b[i].d_txns;
        a.ops = reinterpret_cast<const uint64_t*>(b[i].d_ops);
        a.operands = reinterpret_cast<const ulonglong2*>(b[i].d_operands);
        a.n_txns = b[i].n_txns;
        a.n_ops = b[i].n_ops;
        a.results = b[i].d_results;
        a.reads = reinterpret_cast<ulonglong2*>(b[i].d_reads);
        a.table = db->table;
        a.n_records = db->d.n_records;
        a.n_fields = db->d.n_fields;
        a.meta = db->meta;
        a.n_meta = db->n_meta;
        a.order_key = db->order_key;
        a.order_key_uses_base = scheme != GCC_NO_WAIT_2PL;
        a.st = db->st;
        a.dbs = reinterpret_cast<gcc::DbState*>(reinterpret_cast<char*>(pl->d_ms) +
                                                offsetof(gcc::MultiState, clock));
        a.lanes = p.lanes_per_txn;
        a.max_ops = max_ops;
        a.collapse = p.collapse;
        a.backoff_base_ns = p.immediate_restart ? 0u : p.backoff_base_ns;
        a.backoff_cap_ns = p.backoff_cap_ns;
        a.max_attempts = p.max_attempts;
        a.read_retries = p.read_retries;
        a.inject_ppm = p.inject_abort_ppm;
        a.wait_budget_ns = p.wait_budget_ns;
        a.deadline_ns = p.deadline_ns;
        a.seed = p.seed ^ (0x9E3779B97F4A7C15ull * (i + 1));
        a.rq = (p.retry_queue == 2 || p.immediate_restart) ? nullptr : db->rq;
        a.rq_mask = gcc::RETRY_QUEUES - 1;
        a.queue_turn_ns = p.queue_turn_ns;
        a.queue_width = p.queue_width;
        a.queue_after = queue_after_for(p, scheme);
        a.seq = db->fold_flags;                  // TicToc: sequence numbers
        a.mv_wts = db->sort.k0;                  // MVCC: the database's version store
        a.mv_next = db->sort.v0;
        a.mv_field = db->sort.k1;
        a.mv_rec = db->sort.v1;
        a.mv_val = static_cast<ulonglong2*>(db->fold_seg);
        a.mv_slot = db->mv_slot;
        if (scheme == GCC_DET) {
            // the database's own scratch and staging limit, as a plain launch
            a.max_ops = db->d.max_ops_per_txn;
            a.need = db->need;
            a.order_key_uses_base = 0;
            continue;                    // control words are not used
        }
        // control words in a state this scheme can start from
        if ((s = prepare_meta(db, scheme, pl->stream))) return bail(s);
        db->meta_state = state_after(scheme);
    }
    pl->h_args = args;
    if (scheme == GCC_DET) {
        const uint32_t k = std::min<uint32_t>(n, 8);
        pl->side.assign(k, nullptr);
        pl->ev.assign(k + 1, nullptr);
        for (auto& st2 : pl->side)
            if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess)
                return bail(fail(GCC_ERR_CUDA, "cannot create stream"));
        for (auto& e : pl->ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return bail(fail(GCC_ERR_CUDA, "cannot create event"));
        *out = pl;
        return GCC_OK;
    }
    gcc::MultiState ms{};
    ms.total = total;
    {
        const uint64_t chunks = (total + (1u << gcc::FETCH_CHUNK_BITS) - 1) >> gcc::FETCH_CHUNK_BITS;
        unsigned bits = 0;
        while ((1ull << bits) < chunks) ++bits;
        ms.chunk_bits = bits;
        ms.padded = (1ull << bits) << gcc::FETCH_CHUNK_BITS;
    }
    if (cudaMemcpy(pl->d_args, args.data(), sizeof(gcc::ExecArgs) * n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(pl->d_prefix, prefix.data(), sizeof(uint32_t) * (n + 1), cudaMemcpyHostToDevice) ||
        cudaMemcpy(pl->d_own, own.data(), sizeof(gcc::DbState*) * n, cudaMemcpyHostToDevice) ||
        cudaMemcpy(pl->d_ms, &ms, sizeof ms, cudaMemcpyHostToDevice) ||
        cudaStreamSynchronize(pl->stream))
        return bail(fail(GCC_ERR_CUDA, "cannot upload the plan"));

    pl->block = (int)p.warps_per_block * 32;
    const uint32_t slots = pl->block / p.lanes_per_txn;
    pl->smem = (size_t)slots * max_ops * gcc::STAGE_BYTES_PER_OP;
    const int occ = gcc::occupancy_for(scheme, fb, pl->block, pl->smem);
    if (occ <= 0) return bail(fail(GCC_ERR_INVALID, "launch shape does not fit an SM"));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = p.blocks_per_sm ? std::min<int>(p.blocks_per_sm, occ) : occ;
    pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm,
                                                           ((int64_t)total + slots - 1) / slots));
    *out = pl;
    return GCC_OK;
}

gcc_status gcc_multi_launch(gcc_multi_plan* pl, int use_graph, void* stream) {
    if (!pl) return fail(GCC_ERR_INVALID, "null plan");
    if (cudaSetDevice(pl->device) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    for (gcc_db* db : pl->dbs)
        if (pl->scheme != GCC_DET && db->meta_state != META_ZERO &&
            db->meta_state != state_after(pl->scheme))
            return fail(GCC_ERR_INVALID, "a database ran another scheme since the plan was made");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : pl->stream;
    if (!use_graph) return enqueue(pl, st);
    if (!pl->graph) {
        // capture the whole launch sequence once on the plan's own stream
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(pl->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(GCC_ERR_CUDA, "cannot begin stream capture");
        gcc_status s = enqueue(pl, pl->stream);
        const cudaError_t ec = cudaStreamEndCapture(pl->stream, &g);
        if (s) { if (g) cudaGraphDestroy(g); return s; }
        if (ec != cudaSuccess) return fail(GCC_ERR_CUDA, "capture failed: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&pl->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) return fail(GCC_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ei));
    }
    if (cudaGraphLaunch(pl->graph, st) != cudaSuccess) return fail(GCC_ERR_CUDA, "graph launch failed");
    return GCC_OK;
}

gcc_status gcc_multi_stats(gcc_multi_plan* pl, uint32_t i, gcc_batch_stats* stats) {
    if (!pl || !stats || i >= pl->n) return fail(GCC_ERR_INVALID, "bad plan, index or output");
    if (cudaSetDevice(pl->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(GCC_ERR_CUDA, "synchronisation failed");
    gcc::BatchState h{};
    if (cudaMemcpy(&h, pl->dbs[i]->st, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(GCC_ERR_CUDA, "cannot read batch state");
    *stats = gcc_batch_stats{};
    stats->n_txns = pl->h_prefix[i + 1] - pl->h_prefix[i];
    stats->committed = h.committed;
    stats->aborts = h.aborts;
    stats->timeouts = h.timeouts;
    stats->invalid = h.invalid;
    stats->max_attempts = h.max_attempts;
    stats->atomics = h.atomics;
    stats->device_error = h.error;
    stats->scheme = pl->scheme;
    stats->kernel_launches = pl->launches;
    stats->grid_blocks = (uint32_t)pl->grid;
    return GCC_OK;
}

gcc_status gcc_multi_plan_destroy(gcc_multi_plan* pl) {
    if (pl) free_plan(pl);
    return GCC_OK;
}

}  // extern "C"
