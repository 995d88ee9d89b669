// Fused single-pass step (placeholder until the fused kernel lands).
#include "lbm_internal.h"

namespace lbm {

bool fused_supported(const HostPhys &) { return false; }

cudaError_t launch_step_fused(const HostPhys &, const void *, void *, cudaStream_t, cudaEvent_t *)
{
    return cudaErrorNotSupported;
}

}  // namespace lbm
