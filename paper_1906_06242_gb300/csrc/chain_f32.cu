// Fused chain kernels for float kinematic columns.
#include "chain_kernel.cuh"

namespace hepacc {
namespace chain {

hepacc_status run_f32(const LaunchArgs& a) { return run_typed<float>(a); }

unsigned int tu_error_f32(bool clear) {
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
