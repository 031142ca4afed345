// Batched (many-sample) fused chain kernels for __nv_bfloat16 kinematic columns.
#include "chain_kernel.cuh"

namespace hepacc {
namespace chain {

hepacc_status run_batched_bf16(const LaunchArgs& a) {
    if (a.btag_type != HEPACC_F16) return fail(HEPACC_ERR_DTYPE, "batched launches: btag must be F16 with this kinematic type");
    return run_batched_typed<__nv_bfloat16, __half>(a);
}

}  // namespace chain
}  // namespace hepacc
