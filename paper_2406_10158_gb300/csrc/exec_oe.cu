// exec_oe.cu -- execute an order-entry batch (NewOrder / Payment).
#include "engine.cuh"

namespace gcc {

cudaError_t launch_oe_exec(gcc_scheme, const ExecArgs&, int, int, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

int oe_exec_occupancy(gcc_scheme, int, size_t) { return 1; }

}  // namespace gcc
