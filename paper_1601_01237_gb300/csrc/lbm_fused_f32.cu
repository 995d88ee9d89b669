// Instances of the fused step for the f32 storage format.
#include "lbm_fused_impl.cuh"

namespace lbm {
namespace fused {
template cudaError_t fused_t<ST_F32>(const HostPhys &, const void *, void *, cudaStream_t, cudaEvent_t *,
                                  void *);
}  // namespace fused
}  // namespace lbm
