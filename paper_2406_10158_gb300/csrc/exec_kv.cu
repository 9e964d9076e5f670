// exec_kv.cu -- launchers of the key-value execute kernels (the workload
// policy is in kv_work.cuh).
#include "kv_work.cuh"

namespace gcc {

cudaError_t launch_kv_exec(gcc_scheme scheme, uint32_t fb, const ExecArgs& a, int grid,
                           int block, size_t smem, cudaStream_t s) {
#define GCC_KV_CASE(SC)                                                           \
    case SC:                                                                      \
        return fb == 16 ? launch_exec<SC, KvWork<16>>(a, grid, block, smem, s)    \
                        : launch_exec<SC, KvWork<8>>(a, grid, block, smem, s);
    switch (scheme) {
        GCC_KV_CASE(GCC_NO_WAIT_2PL)
        GCC_KV_CASE(GCC_TO)
        GCC_KV_CASE(GCC_OCC)
        GCC_KV_CASE(GCC_DET)
        GCC_KV_CASE(GCC_TICTOC)
        GCC_KV_CASE(GCC_2PL_WAIT_DIE)
        GCC_KV_CASE(GCC_MVCC)
    }
#undef GCC_KV_CASE
    return cudaErrorInvalidValue;
}

int kv_exec_occupancy(gcc_scheme scheme, uint32_t fb, int block, size_t smem) {
#define GCC_KV_OCC(SC)                                                          \
    case SC:                                                                    \
        return fb == 16 ? exec_occupancy<SC, KvWork<16>>(block, smem)           \
                        : exec_occupancy<SC, KvWork<8>>(block, smem);
    switch (scheme) {
        GCC_KV_OCC(GCC_NO_WAIT_2PL)
        GCC_KV_OCC(GCC_TO)
        GCC_KV_OCC(GCC_OCC)
        GCC_KV_OCC(GCC_DET)
        GCC_KV_OCC(GCC_TICTOC)
        GCC_KV_OCC(GCC_2PL_WAIT_DIE)
        GCC_KV_OCC(GCC_MVCC)
    }
#undef GCC_KV_OCC
    return 0;
}

}  // namespace gcc
