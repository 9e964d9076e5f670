// mvcc.cu -- end of a multi-version batch: the newest versions go into the
// table.
//
// During an MVCC batch the table holds every slot's oldest version and the
// batch's committed writes live in the version store, each slot's entries
// linked from its version pointer, newest first (exec_common.cuh, "MVCC").
// After the execute kernel one thread per store entry checks whether it is
// its slot's newest (the slot's version pointer names it); if so it writes
// its value into the table slot and clears the pointer.  The record heads are
// then zeroed, so the next batch starts from one version per slot, no
// pointers and empty heads.  Work: one pass over the entries (one per write
// of a transaction that attempted) and one over the heads.
#include "engine.cuh"

namespace gcc {
namespace {

template <int FB>
__global__ void mv_flatten_kernel(const __grid_constant__ ExecArgs a) {
    const unsigned long long used = a.st->mv_used;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < used; i += stride) {
        // a transaction that gave up left its range of entries unwritten
        // (stale scratch): no version pointer names them, but their record
        // and field must be checked before they are used as an index
        const uint32_t r = a.mv_rec[i], f = a.mv_field[i];
        if (r >= a.n_records || f >= a.n_fields) continue;
        uint32_t* p = a.mv_slot + (uint64_t)f * a.n_records + r;
        if (*p != i + 1) continue;                 // an older version of its slot
        uint8_t* slot = a.table + ((uint64_t)f * a.n_records + r) * FB;
        const ulonglong2 v = a.mv_val[i];
        if (FB == 16) st_slot16(slot, v);
        else st_relaxed(reinterpret_cast<uint64_t*>(slot), v.x);
        *p = 0;
    }
}

}  // namespace

cudaError_t launch_mv_flatten(const ExecArgs& a, uint32_t field_bytes, cudaStream_t st) {
    const uint64_t blocks = (a.n_ops + 255) / 256;
    if (blocks) {
        if (field_bytes == 16) mv_flatten_kernel<16><<<(unsigned)blocks, 256, 0, st>>>(a);
        else mv_flatten_kernel<8><<<(unsigned)blocks, 256, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(a.meta, 0, (size_t)a.n_meta * 16, st);
    return e;
}

}  // namespace gcc
