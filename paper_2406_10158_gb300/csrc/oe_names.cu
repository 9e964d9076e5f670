// oe_names.cu -- payment by customer last name: the per-district secondary
// index and the resolution of by-name ops.
//
// The paper's GPU index is a sorted array searched by binary search
// (Sec. III-D, "Index"); the payment transaction it studies (Sec. IV-A)
// names its customer by id or, in the TPC-C mix, by last name.  Here the
// names are two never-written int64 columns (c_last, c_first).  Per district
// the customers are sorted by (last name, first name, index); the index holds
// the sorted customer numbers and, beside them, their last names.  A by-name
// op (key = the customer's district, aux = the last-name id) is resolved
// before any control word is touched: binary searches bound the name's run,
// and the customer at position ceil(n/2) of the run is the one paid -- the
// op becomes an ordinary payment of that customer.  Names never change during
// a batch, so resolving every op up front gives the same customer as
// resolving it inside the transaction, in any serial order.
#include "engine.cuh"

namespace gcc {
namespace {

constexpr uint32_t CUST = 3000;

// One block per district: each customer's place in (last, first, index)
// order is the number of the district's customers before it.
__global__ void __launch_bounds__(1024)
name_index_kernel(const int64_t* __restrict__ c_last, const int64_t* __restrict__ c_first,
                  uint32_t* __restrict__ idx, int64_t* __restrict__ last_sorted) {
    __shared__ int64_t sl[CUST];
    __shared__ int64_t sf[CUST];
    const uint64_t base = (uint64_t)blockIdx.x * CUST;
    for (uint32_t c = threadIdx.x; c < CUST; c += blockDim.x) {
        sl[c] = c_last[base + c];
        sf[c] = c_first[base + c];
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < CUST; c += blockDim.x) {
        const int64_t l = sl[c], f = sf[c];
        uint32_t rank = 0;
        for (uint32_t o = 0; o < CUST; ++o)
            rank += (sl[o] < l) || (sl[o] == l && (sf[o] < f || (sf[o] == f && o < c)));
        idx[base + rank] = c;
        last_sorted[base + rank] = l;
    }
}

// First position in [lo, hi) whose name is not below `name` (upper: above).
__device__ __forceinline__ uint32_t name_bound(const int64_t* s, uint32_t lo, uint32_t hi,
                                               int64_t name, bool upper) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const int64_t v = s[mid];
        if (upper ? v <= name : v < name) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void resolve_kernel(const uint64_t* __restrict__ ops, uint64_t n, uint32_t W,
                               const uint32_t* __restrict__ idx,
                               const int64_t* __restrict__ last_sorted,
                               uint64_t* __restrict__ out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t d = ops[i];
    if (((d >> 40) & 0xffu) == GCC_OE_C_PAY_BY_NAME) {
        const uint32_t district = (uint32_t)d;
        const int64_t name = (int64_t)(d >> 48);
        uint64_t r = (uint64_t)0xffu << 40;        // an unknown kind: the txn is invalid
        if (district < 10u * W) {
            const uint64_t base = (uint64_t)district * CUST;
            const int64_t* s = last_sorted + base;
            const uint32_t lo = name_bound(s, 0, CUST, name, false);
            const uint32_t hi = name_bound(s, lo, CUST, name, true);
            if (hi > lo) {
                const uint32_t c = idx[base + lo + (hi - lo + 1) / 2 - 1];
                r = (uint64_t)(uint32_t)(base + c) | ((uint64_t)GCC_OE_C_PAY << 40);
            }
        }
        d = r;
    }
    out[i] = d;
}

}  // namespace

cudaError_t build_name_index(const int64_t* c_last, const int64_t* c_first, uint32_t n_districts,
                             uint32_t* idx, int64_t* last_sorted, cudaStream_t st) {
    if (n_districts == 0) return cudaSuccess;
    name_index_kernel<<<n_districts, 1024, 0, st>>>(c_last, c_first, idx, last_sorted);
    return cudaGetLastError();
}

cudaError_t resolve_by_name(const uint64_t* ops, uint64_t n, uint32_t W, const uint32_t* idx,
                            const int64_t* last_sorted, uint64_t* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    resolve_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ops, n, W, idx, last_sorted, out);
    return cudaGetLastError();
}

}  // namespace gcc
