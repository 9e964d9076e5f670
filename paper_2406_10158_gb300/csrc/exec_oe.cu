// exec_oe.cu -- the execute kernel instantiated for the order-entry workload.
#include "oe_work.cuh"

namespace gcc {

using oe::OeWork;

cudaError_t launch_oe_exec(gcc_scheme scheme, const ExecArgs& a, int grid, int block, size_t smem,
                           cudaStream_t s) {
    switch (scheme) {
        case GCC_NO_WAIT_2PL: return launch_exec<GCC_NO_WAIT_2PL, OeWork>(a, grid, block, smem, s);
        case GCC_TO: return launch_exec<GCC_TO, OeWork>(a, grid, block, smem, s);
        case GCC_OCC: return launch_exec<GCC_OCC, OeWork>(a, grid, block, smem, s);
        case GCC_DET: return launch_exec<GCC_DET, OeWork>(a, grid, block, smem, s);
        case GCC_TICTOC: return launch_exec<GCC_TICTOC, OeWork>(a, grid, block, smem, s);
        case GCC_2PL_WAIT_DIE: return launch_exec<GCC_2PL_WAIT_DIE, OeWork>(a, grid, block, smem, s);
        default: break;   // GCC_MVCC: key-value only
    }
    return cudaErrorInvalidValue;
}

int oe_exec_occupancy(gcc_scheme scheme, int block, size_t smem) {
    switch (scheme) {
        case GCC_NO_WAIT_2PL: return exec_occupancy<GCC_NO_WAIT_2PL, OeWork>(block, smem);
        case GCC_TO: return exec_occupancy<GCC_TO, OeWork>(block, smem);
        case GCC_OCC: return exec_occupancy<GCC_OCC, OeWork>(block, smem);
        case GCC_DET: return exec_occupancy<GCC_DET, OeWork>(block, smem);
        case GCC_TICTOC: return exec_occupancy<GCC_TICTOC, OeWork>(block, smem);
        case GCC_2PL_WAIT_DIE: return exec_occupancy<GCC_2PL_WAIT_DIE, OeWork>(block, smem);
        default: break;
    }
    return 0;
}

}  // namespace gcc
