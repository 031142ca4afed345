// Fused chain kernels (compacting form) for float16 kinematic columns.
#include "fused_kernel.cuh"

namespace hepacc {
namespace fused {

hepacc_status run_fused_f16(const FusedArgs& a) { return run_fused_typed<__half>(a); }

}  // namespace fused
}  // namespace hepacc
