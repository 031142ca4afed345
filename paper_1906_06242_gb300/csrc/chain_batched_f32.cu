// Batched (many-sample) fused chain kernels for float kinematic columns.
#include "chain_kernel.cuh"

namespace hepacc {
namespace chain {

hepacc_status run_batched_f32(const LaunchArgs& a) {
    if (a.btag_type != HEPACC_F32) return fail(HEPACC_ERR_DTYPE, "batched launches: btag must be F32 with this kinematic type");
    return run_batched_typed<float, float>(a);
}

}  // namespace chain
}  // namespace hepacc
