// Fused chain kernels (compacting form) for bfloat16 kinematic columns.
#include "fused_kernel.cuh"

namespace hepacc {
namespace fused {

hepacc_status run_fused_bf16(const FusedArgs& a) { return run_fused_typed<__nv_bfloat16>(a); }

}  // namespace fused
}  // namespace hepacc
