// seeded_init.cu -- fill a key-value table with its seeded initial values on
// the device (the values of seeded_init.cuh), one slot per thread and pass of
// a grid-stride loop, in the table's field-major order so that consecutive
// threads write consecutive slots.
#include <algorithm>

#include "engine.cuh"
#include "seeded_init.cuh"

namespace gcc {
namespace {

template <int FB>
__global__ void seeded_init_kernel(uint8_t* __restrict__ table, uint64_t n_records,
                                   uint32_t n_fields, uint64_t seed) {
    const uint64_t n = n_records * n_fields;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const uint64_t field = s / n_records, key = s - field * n_records;
        const uint64_t lo = seeded::slot_lo(seed, key, field, n_fields);
        if constexpr (FB == 8) {
            reinterpret_cast<uint64_t*>(table)[s] = lo;
        } else {
            reinterpret_cast<ulonglong2*>(table)[s] =
                make_ulonglong2(lo, seeded::slot_hi(seed, key, field, n_fields));
        }
    }
}

}  // namespace

cudaError_t launch_seeded_init(uint8_t* table, uint64_t n_records, uint32_t n_fields,
                               uint32_t field_bytes, uint64_t seed, int sm_count,
                               cudaStream_t st) {
    const uint64_t n = n_records * n_fields;
    if (n == 0) return cudaSuccess;
    const int block = 256;
    const uint64_t blocks = (n + block - 1) / block;
    const unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)std::max(sm_count, 1) * 8);
    if (field_bytes == 16)
        seeded_init_kernel<16><<<grid, block, 0, st>>>(table, n_records, n_fields, seed);
    else
        seeded_init_kernel<8><<<grid, block, 0, st>>>(table, n_records, n_fields, seed);
    return cudaGetLastError();
}

}  // namespace gcc
