// occ_group.cu -- group commit for OCC key-value batches: forming the units
// before the launch, and the launchers of the group-commit kernel.
//
// Units: every transaction is keyed by the record, among those it writes,
// with the most writes in the batch (ties: the lower record), if that record
// has at least `min_writes` writes and every other record the transaction
// reads or writes has fewer; by none otherwise (a member with a second
// contended record would often fail while its unit holds the key, and units
// whose members share several contended records keep failing one another).
// A stable radix sort of the transaction ids by key puts each key's
// transactions in id order; each key's run is cut into units of U
// consecutive transactions.
// Each transaction gets one link word: the next member of its unit (or none),
// and whether it follows a lower id of the same unit.  Transactions keyed by
// none run alone.
#include "kv_work.cuh"
#include "occ_group.cuh"

namespace gcc {
namespace {

inline unsigned blocks_of(uint64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// per-record write counts of the batch
__global__ void unit_hist(const uint64_t* __restrict__ ops, uint64_t n, uint64_t n_records,
                          uint32_t* __restrict__ cnt) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t d = ops[i];
    if (op_kind(d) == GCC_OP_ADD && op_key(d) < n_records) atomicAdd(&cnt[op_key(d)], 1u);
}

// each transaction's key: its most-written record, or none_key
__global__ void unit_keys(const gcc_txn* __restrict__ txns, uint32_t n_txns,
                          const uint64_t* __restrict__ ops, uint64_t n_ops, uint64_t n_records,
                          uint32_t max_ops, const uint32_t* __restrict__ cnt, uint32_t min_writes,
                          uint32_t none_key, uint32_t* __restrict__ keys, uint32_t* __restrict__ ids) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_txns) return;
    const gcc_txn tx = txns[t];
    uint32_t best = none_key, bc = 0, second = 0;
    if (tx.n_ops <= max_ops && tx.first_op + tx.n_ops <= n_ops) {
        for (uint32_t j = 0; j < tx.n_ops; ++j) {
            const uint64_t d = ops[tx.first_op + j];
            if (op_key(d) >= n_records) continue;
            const uint32_t c = cnt[op_key(d)];
            if (op_kind(d) == GCC_OP_ADD && (c > bc || (c == bc && op_key(d) < best))) {
                if (best != none_key && bc > second) second = bc;
                bc = c;
                best = op_key(d);
            } else if (c > second) {
                second = c;
            }
        }
    }
    keys[t] = (bc >= min_writes && second < min_writes) ? best : none_key;
    ids[t] = t;
}

// link words from the sorted (key, id) order
__global__ void unit_links(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                           uint32_t n, uint32_t U, uint32_t none_key, uint32_t* __restrict__ link) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t k = sk[p], t = sv[p];
    if (k == none_key) { link[t] = UNIT_NONE; return; }
    uint32_t lo = 0, hi = p;                     // first position of key k
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (sk[mid] < k) lo = mid + 1; else hi = mid;
    }
    const uint32_t r = (p - lo) % U;
    const bool next = r != U - 1 && p + 1 < n && sk[p + 1] == k;
    link[t] = (r ? UNIT_FOLLOWER : 0u) | (next ? sv[p + 1] : UNIT_NONE);
}

}  // namespace

uint32_t occ_form_units_launches(uint64_t n_records) {
    int bits = 0;
    for (uint64_t v = n_records; v; v >>= 1) ++bits;
    return 1 + 1 + 1 + 3 * (uint32_t)((bits + 7) / 8) + 1;
}

cudaError_t occ_form_units(const ExecArgs& a, uint32_t* cnt, SortScratch& s, uint32_t* link,
                           uint32_t U, uint32_t min_writes, cudaStream_t st) {
    if (a.n_txns == 0) return cudaSuccess;
    const uint32_t none_key = (uint32_t)a.n_records;   // above every key
    int bits = 0;
    for (uint64_t v = none_key; v; v >>= 1) ++bits;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)a.n_records * 4, st);
    if (e != cudaSuccess) return e;
    if (a.n_ops) unit_hist<<<blocks_of(a.n_ops, 256), 256, 0, st>>>(a.ops, a.n_ops, a.n_records, cnt);
    unit_keys<<<blocks_of(a.n_txns, 256), 256, 0, st>>>(a.txns, a.n_txns, a.ops, a.n_ops,
                                                        a.n_records, a.max_ops, cnt, min_writes,
                                                        none_key, s.k0, s.v0);
    uint32_t *sk = nullptr, *sv = nullptr;
    if ((e = radix_sort_pairs(s, a.n_txns, bits, &sk, &sv, st)) != cudaSuccess) return e;
    unit_links<<<blocks_of(a.n_txns, 256), 256, 0, st>>>(sk, sv, a.n_txns, U, none_key, link);
    return cudaGetLastError();
}

size_t occ_group_stage_bytes(uint32_t U, uint32_t max_ops) {
    return UnitLayout(U, max_ops).bytes();
}

template <class Work>
static cudaError_t launch_group(const ExecArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
    auto k = occ_group_kernel<Work>;
    if (smem > 40 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_kv_occ_group(uint32_t fb, const ExecArgs& a, int grid, int block, size_t smem,
                                cudaStream_t s) {
    return fb == 16 ? launch_group<KvWork<16>>(a, grid, block, smem, s)
                    : launch_group<KvWork<8>>(a, grid, block, smem, s);
}

int kv_occ_group_occupancy(uint32_t fb, int block, size_t smem) {
    return fb == 16 ? occupancy_of(occ_group_kernel<KvWork<16>>, block, smem)
                    : occupancy_of(occ_group_kernel<KvWork<8>>, block, smem);
}

}  // namespace gcc
