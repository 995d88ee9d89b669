// Instances of the fused step for the f16rel storage format.
#include "lbm_fused_impl.cuh"

namespace lbm {
namespace fused {
template cudaError_t fused_t<ST_F16_REL>(const HostPhys &, const void *, void *, cudaStream_t, cudaEvent_t *,
                                  void *);
}  // namespace fused
}  // namespace lbm
