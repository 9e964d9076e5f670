// det_fold.cu -- the deterministic scheme on key-value batches, by prefix sums.
//
// The deterministic scheme's outcome is the serial execution of the batch in
// transaction-id order (Sec. II-C; Sec. III-E.3 builds the access table the
// same way: (transaction, record) pairs sorted by record).  On a key-value
// batch every op is a READ or an ADD, and ADD is associative and commutative
// (modulo 2^64 on lane 0, modulo 2^16 on bytes 8-9).  So along one slot's
// accesses in transaction-id order, the value an op reads is the slot's
// initial value plus the exclusive prefix sum of the earlier ADD deltas, and
// the final value adds all of them.  This evaluates every record's dependency
// chain with one segmented prefix sum instead of handing the record from op
// to op, which removes the chain latency that dominates under contention.
//
//   validate   one warp per transaction: the same checks as the execute
//              kernel (kinds, keys, fields, distinct keys); invalid
//              transactions are excluded and reported INVALID
//   emit       access table (slot = field * n_records + key, op index)
//   sort       stable radix sort by slot: (slot, transaction id) order
//   deltas     per sorted position the op's delta (0 for READ)
//   scan       segmented exclusive prefix sum of the deltas, tile by tile
//   apply      read value = initial slot value + prefix
//   finals     last access of each slot writes initial + inclusive sum
//   ranks      commit order = rank among valid transactions (= id when all
//              are valid)
#include <algorithm>

#include "engine.cuh"

namespace gcc {
namespace {

constexpr int FB_THREADS = 1024;
constexpr int FB_ITEMS = 4;
constexpr int FB_TILE = FB_THREADS * FB_ITEMS;

__device__ __forceinline__ uint32_t d_key(uint64_t d) { return (uint32_t)d; }
__device__ __forceinline__ uint32_t d_field(uint64_t d) { return (uint32_t)(d >> 32) & 0xffu; }
__device__ __forceinline__ uint32_t d_kind(uint64_t d) { return (uint32_t)(d >> 40) & 0xffu; }

// A running sum in the slot's lane arithmetic.
struct Sum {
    uint64_t lo, hi;       // hi kept modulo 2^16
};
__device__ __forceinline__ Sum sum_add(Sum a, Sum b) {
    return Sum{a.lo + b.lo, (a.hi + b.hi) & 0xFFFFull};
}
// Segmented-scan element: `head` marks the first access of a slot.
struct Seg {
    uint32_t head;
    Sum v;
};
// Scratch of the fold: the tile carries, then one cached delta per op.
size_t fold_carry_bytes(size_t n_ops) {
    return (((n_ops + FB_TILE - 1) / FB_TILE + 1) * sizeof(Seg) + 255) & ~size_t(255);
}
// a followed by b
__device__ __forceinline__ Seg seg_combine(Seg a, Seg b) {
    return Seg{a.head | b.head, b.head ? b.v : sum_add(a.v, b.v)};
}

__device__ __forceinline__ Seg shfl_up_seg(Seg s, int o) {
    Seg r;
    r.head = __shfl_up_sync(0xffffffffu, s.head, o);
    r.v.lo = __shfl_up_sync(0xffffffffu, s.v.lo, o);
    r.v.hi = __shfl_up_sync(0xffffffffu, s.v.hi, o);
    return r;
}

// Block-wide exclusive segmented scan of one element per thread; also
// returns the block's inclusive total.
__device__ Seg block_seg_exclusive(Seg x, Seg* warp_tot, Seg* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    Seg inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Seg up = shfl_up_seg(inc, o);
        if (lane >= o) inc = seg_combine(up, inc);
    }
    Seg exc = shfl_up_seg(inc, 1);
    if (lane == 0) exc = Seg{0u, Sum{0, 0}};
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        Seg w = lane < nw ? warp_tot[lane] : Seg{0u, Sum{0, 0}};
        Seg wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Seg up = shfl_up_seg(wi, o);
            if (lane >= o) wi = seg_combine(up, wi);
        }
        Seg we = shfl_up_seg(wi, 1);
        if (lane == 0) we = Seg{0u, Sum{0, 0}};
        if (lane < nw) warp_tot[lane] = we;
        if (lane == nw - 1) warp_tot[32] = wi;
    }
    __syncthreads();
    const Seg r = seg_combine(warp_tot[warp], exc);
    if (total) *total = warp_tot[32];
    __syncthreads();
    return r;
}

// --- validation and access table ---------------------------------------------
__global__ void fold_validate(const ExecArgs a, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals, uint32_t* __restrict__ valid_flag,
                              uint32_t none) {
    __shared__ uint32_t skeys[32][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    unsigned invalid = 0;
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + wib; t < a.n_txns; t += warps) {
        const gcc_txn tx = a.txns[t];
        const uint32_t nops = tx.n_ops;
        const uint64_t first = tx.first_op;
        bool bad = nops > a.max_ops || nops > 64 || tx.type != GCC_TXN_KV || first + nops > a.n_ops;
        if (!bad) {
            for (uint32_t j = lane; j < nops; j += 32) {
                const uint64_t d = a.ops[first + j];
                skeys[wib][j] = d_key(d);
                if (d_key(d) >= a.n_records || d_field(d) >= a.n_fields ||
                    (d_kind(d) != GCC_OP_READ && d_kind(d) != GCC_OP_ADD))
                    bad = true;
            }
        }
        __syncwarp();
        if (!__any_sync(0xffffffffu, bad)) {
            for (uint32_t j = lane; j < nops; j += 32)
                for (uint32_t i = 0; i < j; ++i)
                    if (skeys[wib][i] == skeys[wib][j]) bad = true;
        }
        bad = __any_sync(0xffffffffu, bad);
        if (first + nops <= a.n_ops) {
            for (uint32_t j = lane; j < nops; j += 32) {
                const uint64_t d = a.ops[first + j];
                keys[first + j] = bad ? none : d_field(d) * (uint32_t)a.n_records + d_key(d);
                vals[first + j] = (uint32_t)(first + j);
            }
        }
        if (lane == 0) {
            valid_flag[t] = bad ? 0u : 1u;
            a.results[t] = bad ? gcc_txn_result{GCC_TXN_INVALID, 0u, ~0ull}
                               : gcc_txn_result{GCC_TXN_COMMITTED, 1u, 0ull};
            invalid += bad;
        }
        __syncwarp();
    }
    if (lane == 0 && invalid) {
        atomicAdd(&a.st->invalid, (unsigned long long)invalid);
        atomicOr(&a.st->error, GCC_DEVERR_INVALID);
    }
}

// Ops not covered by any transaction's range stay out of the access table.
__global__ void fold_fill_none(uint32_t* __restrict__ keys, uint64_t n, uint32_t none) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = none;
}

// --- segmented scan ---------------------------------------------------------
template <int FB>
__device__ __forceinline__ Seg element(const ExecArgs& a, const uint32_t* sk, const uint32_t* sv,
                                       uint64_t p, uint64_t n, uint32_t none) {
    if (p >= n) return Seg{1u, Sum{0, 0}};
    const uint32_t k = sk[p];
    if (k == none) return Seg{1u, Sum{0, 0}};
    const uint32_t head = (p == 0 || sk[p - 1] != k) ? 1u : 0u;
    const uint32_t op = sv[p];
    Sum v{0, 0};
    if (d_kind(a.ops[op]) == GCC_OP_ADD) {
        const ulonglong2 o = a.operands[op];
        v = Sum{o.x, FB == 16 ? (o.y & 0xFFFFull) : 0ull};
    }
    return Seg{head, v};
}

// The same element from the cache fold_tile_totals filled: the op's delta,
// stored in sorted order, so the second pass streams it instead of gathering
// the op and its operand again.
__device__ __forceinline__ Seg cached_element(const uint32_t* sk, const Sum* cache, uint64_t p,
                                              uint64_t n, uint32_t none) {
    if (p >= n) return Seg{1u, Sum{0, 0}};
    const uint32_t k = sk[p];
    if (k == none) return Seg{1u, Sum{0, 0}};
    return Seg{(p == 0 || sk[p - 1] != k) ? 1u : 0u, cache[p]};
}

template <int FB>
__global__ void __launch_bounds__(FB_THREADS)
fold_tile_totals(const ExecArgs a, const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                 uint64_t n, uint32_t none, Seg* __restrict__ tile_tot, Sum* __restrict__ cache) {
    __shared__ Seg warp_tot[33];
    const uint64_t base = (uint64_t)blockIdx.x * FB_TILE + (uint64_t)threadIdx.x * FB_ITEMS;
    Seg acc{0u, Sum{0, 0}};
#pragma unroll
    for (int i = 0; i < FB_ITEMS; ++i) {
        const Seg e = element<FB>(a, sk, sv, base + i, n, none);
        if (base + i < n) cache[base + i] = e.v;
        acc = seg_combine(acc, e);
    }
    Seg total;
    block_seg_exclusive(acc, warp_tot, &total);
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = total;
}

// Exclusive segmented scan of the tile totals (one block, running carry).
__global__ void __launch_bounds__(FB_THREADS)
fold_scan_tiles(Seg* __restrict__ tile_tot, uint32_t ntiles) {
    __shared__ Seg warp_tot[33];
    Seg carry{0u, Sum{0, 0}};
    for (uint32_t base = 0; base < ntiles; base += FB_THREADS) {
        const uint32_t i = base + threadIdx.x;
        const Seg x = i < ntiles ? tile_tot[i] : Seg{0u, Sum{0, 0}};
        Seg total;
        const Seg ex = block_seg_exclusive(x, warp_tot, &total);
        if (i < ntiles) tile_tot[i] = seg_combine(carry, ex);
        carry = seg_combine(carry, total);
    }
}

template <int FB>
__device__ __forceinline__ ulonglong2 slot_load(const ExecArgs& a, uint32_t slot) {
    const uint8_t* p = a.table + (uint64_t)slot * FB;
    if (FB == 16) return *reinterpret_cast<const ulonglong2*>(p);
    return make_ulonglong2(*reinterpret_cast<const uint64_t*>(p), 0ull);
}
template <int FB>
__device__ __forceinline__ ulonglong2 slot_plus(ulonglong2 v, Sum s) {
    if (FB == 16) return make_ulonglong2(v.x + s.lo, (v.y & ~0xFFFFull) | ((v.y + s.hi) & 0xFFFFull));
    return make_ulonglong2(v.x + s.lo, 0ull);
}

// Read values: initial slot value plus the exclusive prefix within the slot.
// A slot whose accesses all lie in this tile also gets its final value here:
// once the block's initial-value loads are done (the barrier), the slot's
// last access writes initial + inclusive sum.  Slots whose accesses began in
// an earlier tile are left to fold_finals, after every tile has loaded.
template <int FB>
__global__ void __launch_bounds__(FB_THREADS)
fold_apply(const ExecArgs a, const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
           uint64_t n, uint32_t none, const Seg* __restrict__ tile_carry,
           const Sum* __restrict__ cache) {
    __shared__ Seg warp_tot[33];
    const uint64_t tile_base = (uint64_t)blockIdx.x * FB_TILE;
    const uint64_t base = tile_base + (uint64_t)threadIdx.x * FB_ITEMS;
    Seg e[FB_ITEMS];
    Seg acc{0u, Sum{0, 0}};
#pragma unroll
    for (int i = 0; i < FB_ITEMS; ++i) {
        e[i] = cached_element(sk, cache, base + i, n, none);
        acc = seg_combine(acc, e[i]);
    }
    Seg run = seg_combine(tile_carry[blockIdx.x], block_seg_exclusive(acc, warp_tot, nullptr));
    const uint32_t before = tile_base > 0 ? sk[tile_base - 1] : none;   // key entering the tile
    ulonglong2 fin[FB_ITEMS];
    bool last[FB_ITEMS];
#pragma unroll
    for (int i = 0; i < FB_ITEMS; ++i) {
        const uint64_t p = base + i;
        const Sum prefix = e[i].head ? Sum{0, 0} : run.v;
        last[i] = false;
        if (p < n && sk[p] != none) {
            const uint32_t k = sk[p];
            const uint32_t op = sv[p];
            const ulonglong2 init = slot_load<FB>(a, k);
            const ulonglong2 rd = slot_plus<FB>(init, prefix);
            a.reads[op] = rd;
            if ((p + 1 >= n || sk[p + 1] != k) && k != before) {
                fin[i] = slot_plus<FB>(rd, e[i].v);
                last[i] = fin[i].x != init.x || fin[i].y != init.y;   // skip unchanged slots
            }
        }
        run = seg_combine(run, e[i]);
    }
    __syncthreads();                      // every initial value of this tile has been read
#pragma unroll
    for (int i = 0; i < FB_ITEMS; ++i) {
        if (!last[i]) continue;
        uint8_t* dst = a.table + (uint64_t)sk[base + i] * FB;
        if (FB == 16) *reinterpret_cast<ulonglong2*>(dst) = fin[i];
        else *reinterpret_cast<uint64_t*>(dst) = fin[i].x;
    }
}

// The last access of each slot whose accesses began in an earlier tile
// installs the final value (the others were installed by fold_apply).
template <int FB>
__global__ void fold_finals(const ExecArgs a, const uint32_t* __restrict__ sk,
                            const uint32_t* __restrict__ sv, uint64_t n, uint32_t none) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t k = sk[p];
    if (k == none || (p + 1 < n && sk[p + 1] == k)) return;
    const uint64_t tile_base = p / FB_TILE * FB_TILE;
    if (tile_base == 0 || sk[tile_base - 1] != k) return;     // installed by fold_apply
    const uint32_t op = sv[p];
    ulonglong2 v = a.reads[op];                   // initial value + every earlier delta
    if (d_kind(a.ops[op]) == GCC_OP_ADD) {
        const ulonglong2 o = a.operands[op];
        v = slot_plus<FB>(v, Sum{o.x, FB == 16 ? (o.y & 0xFFFFull) : 0ull});
    }
    // only this thread touches the slot now; skip slots that did not change
    const ulonglong2 cur = slot_load<FB>(a, k);
    if (cur.x == v.x && cur.y == v.y) return;
    uint8_t* dst = a.table + (uint64_t)k * FB;
    if (FB == 16) *reinterpret_cast<ulonglong2*>(dst) = v;
    else *reinterpret_cast<uint64_t*>(dst) = v.x;
}

// commit order = rank among valid transactions; counts the commits
__global__ void fold_ranks(const ExecArgs a, const uint32_t* __restrict__ rank, uint32_t n) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (a.results[t].status == GCC_TXN_COMMITTED) a.results[t].commit_order = rank[t];
}

__global__ void fold_count(const ExecArgs a, const uint32_t* __restrict__ rank,
                           const uint32_t* __restrict__ flag, uint32_t n) {
    if (n) {
        a.st->committed = rank[n - 1] + flag[n - 1];
        a.st->max_attempts = a.st->committed ? 1ull : 0ull;
    }
}

inline unsigned blocks_for(uint64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int FB>
cudaError_t fold_run(const ExecArgs& a, SortScratch& s, uint32_t* scan_tmp, uint32_t* flags,
                     void* seg_tmp, cudaStream_t st) {
    const uint64_t n = a.n_ops;
    const uint64_t n_slots = (uint64_t)a.n_fields * a.n_records;
    const uint32_t none = (uint32_t)n_slots;               // sorts after every slot
    int bits = 0;
    for (uint64_t v = n_slots; v; v >>= 1) ++bits;
    if (n) fold_fill_none<<<blocks_for(n, 256), 256, 0, st>>>(s.k0, n, none);
    if (a.n_txns) {
        const int warps_per_block = 8;
        const unsigned grid = std::min<unsigned>(blocks_for(a.n_txns, warps_per_block), 152u * 16u);
        fold_validate<<<grid, warps_per_block * 32, 0, st>>>(a, s.k0, s.v0, flags, none);
    }
    uint32_t *sk = s.k0, *sv = s.v0;
    if (n) {
        cudaError_t e = radix_sort_pairs(s, n, bits, &sk, &sv, st);
        if (e != cudaSuccess) return e;
        const uint32_t ntiles = (uint32_t)((n + FB_TILE - 1) / FB_TILE);
        Seg* tiles = static_cast<Seg*>(seg_tmp);
        Sum* cache = reinterpret_cast<Sum*>(static_cast<char*>(seg_tmp) + fold_carry_bytes(n));
        fold_tile_totals<FB><<<ntiles, FB_THREADS, 0, st>>>(a, sk, sv, n, none, tiles, cache);
        fold_scan_tiles<<<1, FB_THREADS, 0, st>>>(tiles, ntiles);
        fold_apply<FB><<<ntiles, FB_THREADS, 0, st>>>(a, sk, sv, n, none, tiles, cache);
        fold_finals<FB><<<blocks_for(n, 256), 256, 0, st>>>(a, sk, sv, n, none);
    }
    if (a.n_txns) {
        // dense commit order: exclusive count of valid transactions before each
        uint32_t* rank = flags + a.n_txns;
        cudaError_t e = cudaMemcpyAsync(rank, flags, (size_t)a.n_txns * 4,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = exclusive_scan_u32(rank, a.n_txns, scan_tmp, st);
        if (e != cudaSuccess) return e;
        fold_ranks<<<blocks_for(a.n_txns, 256), 256, 0, st>>>(a, rank, a.n_txns);
        fold_count<<<1, 1, 0, st>>>(a, rank, flags, a.n_txns);
    }
    return cudaGetLastError();
}

}  // namespace

size_t fold_seg_bytes(size_t max_ops) {
    return fold_carry_bytes(max_ops) + max_ops * sizeof(Sum);
}

cudaError_t det_fold_kv(const ExecArgs& a, uint32_t field_bytes, SortScratch& s,
                        uint32_t* scan_tmp, uint32_t* flags, void* seg_tmp, cudaStream_t st) {
    return field_bytes == 16 ? fold_run<16>(a, s, scan_tmp, flags, seg_tmp, st)
                             : fold_run<8>(a, s, scan_tmp, flags, seg_tmp, st);
}

}  // namespace gcc
