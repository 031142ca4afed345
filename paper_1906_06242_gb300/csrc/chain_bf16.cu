// Fused chain kernels for __nv_bfloat16 kinematic columns.
#include "chain_kernel.cuh"

namespace hepacc {
namespace chain {

hepacc_status run_bf16(const LaunchArgs& a) { return run_typed<__nv_bfloat16>(a); }

unsigned int tu_error_bf16(bool clear) {
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
