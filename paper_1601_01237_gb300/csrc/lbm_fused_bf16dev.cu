// Instances of the fused step for the bf16dev storage format.
#include "lbm_fused_impl.cuh"

namespace lbm {
namespace fused {
template cudaError_t fused_t<ST_BF16_DEV>(const HostPhys &, const void *, void *, cudaStream_t, cudaEvent_t *,
                                  void *);
}  // namespace fused
}  // namespace lbm
