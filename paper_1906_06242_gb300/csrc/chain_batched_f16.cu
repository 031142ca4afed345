// Batched (many-sample) fused chain kernels for __half kinematic columns.
#include "chain_kernel.cuh"

namespace hepacc {
namespace chain {

hepacc_status run_batched_f16(const LaunchArgs& a) {
    if (a.btag_type != HEPACC_F16) return fail(HEPACC_ERR_DTYPE, "batched launches: btag must be F16 with this kinematic type");
    return run_batched_typed<__half, __half>(a);
}

unsigned int tu_error_batched_f16(bool clear) {
    unsigned int v = 0;
    cudaMemcpyFromSymbol(&v, g_device_error, sizeof v);
    if (clear && v) {
        unsigned int z = 0;
        cudaMemcpyToSymbol(g_device_error, &z, sizeof z);
    }
    return v;
}

}  // namespace chain
}  // namespace hepacc
