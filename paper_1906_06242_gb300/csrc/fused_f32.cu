// Fused chain kernels (compacting form) for float kinematic columns.
#include "fused_kernel.cuh"

namespace hepacc {
namespace fused {

hepacc_status run_fused_f32(const FusedArgs& a) { return run_fused_typed<float>(a); }

}  // namespace fused
}  // namespace hepacc
