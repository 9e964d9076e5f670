// order.cu -- ordering kernels: radix sort, prefix sum, the deterministic
// scheme's access table, and dense commit ranks.
//
// The deterministic scheme's preprocessing follows Sec. III-E.3: gather the
// (transaction, record) pairs of the batch into an access table, sort it by
// record, and find each record's boundaries with a prefix sum.  Because the
// ops array is in transaction-id order, a stable sort by record alone yields
// (record, transaction id) order.  Each op then gets a wait threshold:
//   writer at sorted position p     -> all ops before it on the record done
//                                      (record's op counter >= p)
//   reader at sorted position p     -> all writes before it on the record done
//                                      (record's write counter >= W[p], W the
//                                      exclusive prefix count of writes)
// and every record's counter word starts at (first position, W[first]).
// This is the dataflow form of executing the conflict graph rank by rank
// (Sec. II-C): an op runs as soon as its conflicting predecessors have run.
#include "engine.cuh"

namespace gcc {
namespace {

constexpr int RS_BLOCK = 256;
constexpr int RS_CHUNKS = 8;
constexpr int RS_TILE = RS_BLOCK * RS_CHUNKS;
constexpr int RS_WARPS = RS_BLOCK / 32;

__device__ __forceinline__ unsigned lt_mask() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a block of 32*NW threads.
template <int NW>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < NW ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (warp ? warp_sums[warp - 1] : 0) + x - v;
    if (total) *total = warp_sums[NW - 1];
    __syncthreads();
    return before;
}

// --- radix sort --------------------------------------------------------------
__global__ void rs_hist(const uint32_t* __restrict__ keys, size_t n, int shift,
                        uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * RS_TILE;
    for (int c = 0; c < RS_CHUNKS; ++c) {
        const size_t i = base + (size_t)c * RS_BLOCK + threadIdx.x;
        const uint32_t dg = i < n ? (keys[i] >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256u && (peers & lt_mask()) == 0) atomicAdd(&h[dg], __popc(peers));
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's per-tile counts.
__global__ void rs_scan_rows(uint32_t* __restrict__ hist, uint32_t ntiles,
                             uint32_t* __restrict__ totals) {
    __shared__ uint32_t warp_sums[32];
    uint32_t* row = hist + (size_t)blockIdx.x * ntiles;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ntiles; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? row[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<32>(v, warp_sums, &tot);
        if (i < ntiles) row[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Stable scatter of one tile.  Each warp ranks its own contiguous run of
// RS_CHUNKS * 32 items with warp-private digit counters (match_any groups the
// lanes of one digit; no block barrier inside the loop); one digit-major
// scan over (digit, warp) then gives every item its position in the tile
// staged in digit order -- warp w's items of a digit follow warp w-1's, which
// keeps the sort stable -- and each digit's run goes to its global position
// with consecutive threads on consecutive addresses (coalesced).
__global__ void __launch_bounds__(RS_BLOCK)
rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, size_t n, int shift,
           const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals,
           uint32_t ntiles) {
    __shared__ uint32_t gbase[256];            // global start of each digit's run for this tile
    __shared__ uint32_t dstart[256];           // start of each digit within the staged tile
    __shared__ uint32_t wc[RS_WARPS][256];     // per-warp digit counts, then per-warp starts
    __shared__ uint32_t skey[RS_TILE];
    __shared__ uint32_t sval[RS_TILE];
    __shared__ uint32_t warp_sums[32];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    gbase[t] = block_exclusive_scan<RS_WARPS>(totals[t], warp_sums, nullptr) +
               hist[(size_t)t * ntiles + blockIdx.x];
    for (int w = 0; w < RS_WARPS; ++w) wc[w][t] = 0;
    __syncthreads();
    const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
    const size_t base = tile0 + (size_t)warp * (RS_CHUNKS * 32);
    uint32_t key[RS_CHUNKS], val[RS_CHUNKS], rank[RS_CHUNKS];
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        const size_t i = base + (size_t)c * 32 + lane;
        const bool valid = i < n;
        key[c] = valid ? kin[i] : 0u;
        val[c] = valid ? vin[i] : 0u;
    }
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        const bool valid = base + (size_t)c * 32 + lane < n;
        const uint32_t dg = valid ? (key[c] >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t prior = valid ? wc[warp][dg] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask()) == 0) wc[warp][dg] = prior + __popc(peers);
        __syncwarp();
        rank[c] = prior + __popc(peers & lt_mask());
    }
    __syncthreads();
    uint32_t tot = 0;                          // thread t owns digit t
    for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t x = wc[w][t];
        wc[w][t] = tot;
        tot += x;
    }
    dstart[t] = block_exclusive_scan<RS_WARPS>(tot, warp_sums, nullptr);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        if (base + (size_t)c * 32 + lane < n) {
            const uint32_t dg = (key[c] >> shift) & 255u;
            const uint32_t pos = dstart[dg] + wc[warp][dg] + rank[c];
            skey[pos] = key[c];
            sval[pos] = val[c];
        }
    }
    __syncthreads();
    const uint32_t tile_n = (uint32_t)((n - tile0) < (size_t)RS_TILE ? (n - tile0) : RS_TILE);
    for (uint32_t i = t; i < tile_n; i += RS_BLOCK) {
        const uint32_t k = skey[i];
        const uint32_t dg = (k >> shift) & 255u;
        const uint32_t out = gbase[dg] + (i - dstart[dg]);
        kout[out] = k;
        vout[out] = sval[i];
    }
}

// --- prefix sum -------------------------------------------------------------
constexpr int SC_BLOCK = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_BLOCK * SC_ITEMS;

__global__ void scan_tile_sums(const uint32_t* __restrict__ d, size_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_sums[32];
    const size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t s = 0;
    for (int k = 0; k < SC_ITEMS; ++k)
        if (base + k < n) s += d[base + k];
    uint32_t tot;
    block_exclusive_scan<32>(s, warp_sums, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums(uint32_t* __restrict__ sums, uint32_t ntiles) {
    __shared__ uint32_t warp_sums[32];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ntiles; base += SC_BLOCK) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? sums[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<32>(v, warp_sums, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
    }
}

__global__ void scan_apply(uint32_t* __restrict__ d, size_t n, const uint32_t* __restrict__ sums) {
    __shared__ uint32_t warp_sums[32];
    const size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t s = 0;
    for (int k = 0; k < SC_ITEMS; ++k) {
        v[k] = base + k < n ? d[base + k] : 0;
        s += v[k];
    }
    uint32_t run = block_exclusive_scan<32>(s, warp_sums, nullptr) + sums[blockIdx.x];
    for (int k = 0; k < SC_ITEMS; ++k) {
        if (base + k < n) d[base + k] = run;
        run += v[k];
    }
}

// --- deterministic scheme ---------------------------------------------------
__global__ void det_emit(const uint64_t* __restrict__ ops, uint64_t n, int schema, uint32_t W,
                         uint32_t none, uint32_t n_meta, uint32_t* __restrict__ keys,
                         uint32_t* __restrict__ vals) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t r = cc_record(ops[i], schema, W, none);
    if (r >= n_meta) r = none;          // malformed ops are rejected by the kernel
    keys[i] = r;
    vals[i] = (uint32_t)i;
}

__global__ void det_flags(const uint64_t* __restrict__ ops, const uint32_t* __restrict__ sv,
                          uint64_t n, uint32_t* __restrict__ flags) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    flags[p] = kind_writes((uint32_t)(ops[sv[p]] >> 40) & 0xffu) ? 1u : 0u;
}

// need: a write (or, when every access conflicts, any op) waits for all
// earlier ops on its record, a read for the earlier writes.
__global__ void det_need(const uint64_t* __restrict__ ops, const uint32_t* __restrict__ sk,
                         const uint32_t* __restrict__ sv, const uint32_t* __restrict__ wpre,
                         uint64_t n, uint32_t none, int all_conflict, uint32_t* __restrict__ need,
                         uint64_t* __restrict__ meta) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t key = sk[p];
    if (key == none) return;
    const uint32_t op = sv[p];
    const bool w = kind_writes((uint32_t)(ops[op] >> 40) & 0xffu);
    need[op] = (w || all_conflict) ? (uint32_t)p : wpre[p];
    if (p == 0 || sk[p - 1] != key) meta[key] = ((uint64_t)p << 32) | wpre[p];
}

// --- dense commit ranks -------------------------------------------------------
// Sort keys are 32-bit offsets from the batch's starting clock, all-ones
// marking transactions that did not commit; a batch that used more
// timestamps than that reports GCC_DEVERR_TS_OVERFLOW.
__global__ void dense_emit(const gcc_txn_result* __restrict__ res,
                           const unsigned long long* __restrict__ okey,
                           BatchState* __restrict__ st, int use_base, uint32_t n,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long base = use_base ? st->ticket_base : 0ull;
    uint32_t k = 0xffffffffu;
    if (res[t].status == GCC_TXN_COMMITTED) {
        const unsigned long long d = okey[t] - base;
        if (d >= 0xffffffffull) atomicOr(&st->error, GCC_DEVERR_TS_OVERFLOW);
        k = (uint32_t)d;
    }
    keys[t] = k;
    vals[t] = t;
}

__global__ void dense_rank(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                           uint32_t n, gcc_txn_result* __restrict__ res) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || sk[p] == 0xffffffffu) return;
    res[sv[p]].commit_order = p;
}

// TicToc's serial order, (timestamp, sequence number), by three stable 32-bit
// sorts: sequence number, then the timestamp's low and high words.  Pass 0
// keys each transaction by its sequence number; passes 1 and 2 re-key the
// sorted order by a timestamp word.  Transactions that did not commit carry
// all-ones keys and stay last.
__global__ void tt_emit(const gcc_txn_result* __restrict__ res,
                        const unsigned long long* __restrict__ okey,
                        const uint32_t* __restrict__ seq, const uint32_t* __restrict__ sv,
                        int pass, uint32_t n, uint32_t* __restrict__ keys,
                        uint32_t* __restrict__ vals) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t t = pass == 0 ? p : sv[p];
    const bool c = res[t].status == GCC_TXN_COMMITTED;
    uint32_t k = 0xffffffffu;
    if (c) k = pass == 0 ? seq[t] : pass == 1 ? (uint32_t)okey[t] : (uint32_t)(okey[t] >> 32);
    keys[p] = k;
    vals[p] = t;
}

// Deterministic scheme run op by op: every committed transaction's position
// among the committed ones in id order (an invalid transaction takes none).
__global__ void id_rank_emit(const gcc_txn_result* __restrict__ res, uint32_t n,
                             uint32_t* __restrict__ flags) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) flags[t] = res[t].status == GCC_TXN_COMMITTED ? 1u : 0u;
}

__global__ void id_rank_apply(const uint32_t* __restrict__ before, uint32_t n,
                              gcc_txn_result* __restrict__ res) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && res[t].status == GCC_TXN_COMMITTED) res[t].commit_order = before[t];
}

__global__ void batch_begin_kernel(BatchState* st, DbState* dbs, int scheme) {
    BatchState z{};
    z.ticket_base = scheme == GCC_TO ? dbs->to_clock : dbs->occ_clock;
    *st = z;
}

inline unsigned blocks_for(uint64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

size_t sort_max_tiles(size_t n) { return (n + RS_TILE - 1) / RS_TILE; }

cudaError_t radix_sort_pairs(SortScratch& s, size_t n, int bits, uint32_t** keys_out,
                             uint32_t** vals_out, cudaStream_t st) {
    uint32_t *ki = s.k0, *vi = s.v0, *ko = s.k1, *vo = s.v1;
    if (n == 0) { *keys_out = ki; *vals_out = vi; return cudaSuccess; }
    const uint32_t ntiles = (uint32_t)sort_max_tiles(n);
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist<<<ntiles, RS_BLOCK, 0, st>>>(ki, n, shift, s.hist, ntiles);
        rs_scan_rows<<<256, 1024, 0, st>>>(s.hist, ntiles, s.totals);
        rs_scatter<<<ntiles, RS_BLOCK, 0, st>>>(ki, vi, ko, vo, n, shift, s.hist, s.totals, ntiles);
        uint32_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    *keys_out = ki;
    *vals_out = vi;
    return cudaGetLastError();
}

size_t scan_tmp_words(size_t n) { return (n + SC_TILE - 1) / SC_TILE + 1; }

cudaError_t exclusive_scan_u32(uint32_t* d, size_t n, uint32_t* tmp, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t ntiles = (uint32_t)((n + SC_TILE - 1) / SC_TILE);
    scan_tile_sums<<<ntiles, SC_BLOCK, 0, st>>>(d, n, tmp);
    scan_sums<<<1, SC_BLOCK, 0, st>>>(tmp, ntiles);
    scan_apply<<<ntiles, SC_BLOCK, 0, st>>>(d, n, tmp);
    return cudaGetLastError();
}

cudaError_t det_prepare(const ExecArgs& a, SortScratch& s, uint32_t* scan_tmp, int key_bits,
                        int schema, cudaStream_t st, bool all_conflict) {
    const uint64_t n = a.n_ops;
    if (n == 0) return cudaSuccess;
    const uint32_t none = (uint32_t)a.n_meta;   // sorts after every real record
    det_emit<<<blocks_for(n, 256), 256, 0, st>>>(a.ops, n, schema, a.n_warehouses, none,
                                                 (uint32_t)a.n_meta, s.k0, s.v0);
    uint32_t *sk, *sv;
    cudaError_t e = radix_sort_pairs(s, n, key_bits, &sk, &sv, st);
    if (e != cudaSuccess) return e;
    uint32_t* flags = (sk == s.k0) ? s.k1 : s.k0;   // the free key buffer
    det_flags<<<blocks_for(n, 256), 256, 0, st>>>(a.ops, sv, n, flags);
    e = exclusive_scan_u32(flags, n, scan_tmp, st);
    if (e != cudaSuccess) return e;
    det_need<<<blocks_for(n, 256), 256, 0, st>>>(a.ops, sk, sv, flags, n, none, all_conflict ? 1 : 0,
                                                 const_cast<uint32_t*>(a.need), a.meta);
    return cudaGetLastError();
}

cudaError_t densify_commit_order(const ExecArgs& a, SortScratch& s, cudaStream_t st) {
    const uint32_t n = a.n_txns;
    if (n == 0) return cudaSuccess;
    dense_emit<<<blocks_for(n, 256), 256, 0, st>>>(a.results, a.order_key, a.st,
                                                   a.order_key_uses_base, n, s.k0, s.v0);
    uint32_t *sk, *sv;
    cudaError_t e = radix_sort_pairs(s, n, 32, &sk, &sv, st);
    if (e != cudaSuccess) return e;
    dense_rank<<<blocks_for(n, 256), 256, 0, st>>>(sk, sv, n, a.results);
    return cudaGetLastError();
}

cudaError_t densify_tictoc(const ExecArgs& a, SortScratch& s, cudaStream_t st) {
    const uint32_t n = a.n_txns;
    if (n == 0) return cudaSuccess;
    uint32_t *sk = nullptr, *sv = nullptr;
    for (int pass = 0; pass < 3; ++pass) {
        // the previous pass's sorted values feed the next pass's keys; when the
        // sort left them in (k0, v0), tt_emit rewrites those in place by index
        tt_emit<<<blocks_for(n, 256), 256, 0, st>>>(a.results, a.order_key, a.seq, sv, pass, n,
                                                    s.k0, s.v0);
        cudaError_t e = radix_sort_pairs(s, n, 32, &sk, &sv, st);
        if (e != cudaSuccess) return e;
    }
    dense_rank<<<blocks_for(n, 256), 256, 0, st>>>(sk, sv, n, a.results);
    return cudaGetLastError();
}

cudaError_t densify_in_id_order(const ExecArgs& a, uint32_t* flags, uint32_t* scan_tmp,
                                cudaStream_t st) {
    const uint32_t n = a.n_txns;
    if (n == 0) return cudaSuccess;
    id_rank_emit<<<blocks_for(n, 256), 256, 0, st>>>(a.results, n, flags);
    cudaError_t e = exclusive_scan_u32(flags, n, scan_tmp, st);
    if (e != cudaSuccess) return e;
    id_rank_apply<<<blocks_for(n, 256), 256, 0, st>>>(flags, n, a.results);
    return cudaGetLastError();
}

cudaError_t launch_batch_begin(BatchState* st, DbState* dbs, gcc_scheme scheme, cudaStream_t s) {
    batch_begin_kernel<<<1, 1, 0, s>>>(st, dbs, (int)scheme);
    return cudaGetLastError();
}

}  // namespace gcc
