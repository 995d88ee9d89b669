// Instances of the reverse step for the f32 storage format.
#include "lbm_adjoint_impl.cuh"

namespace lbm {
namespace adj {
template cudaError_t adj_step_t<ST_F32>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
}  // namespace adj
}  // namespace lbm
