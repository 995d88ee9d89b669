// Fused single-pass time step: dispatch over the storage formats.  The kernel
// templates live in lbm_fused_impl.cuh; each storage format is instantiated
// in a translation unit of its own (lbm_fused_<format>.cu), so that they
// compile in parallel.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace fused {
template <int S>
cudaError_t fused_t(const HostPhys &h, const void *fin, void *fout, cudaStream_t s, cudaEvent_t *ev, void *s_out);
}  // namespace fused

bool fused_supported(const HostPhys &p)
{
    // 32-bit offsets of the cell pairs inside the 19 direction arrays; tiles of
    // 32 x 8 columns, chunks of at least 8 planes
    return p.storage != ST_F64 && (long long)Q * p.N < (1LL << 32) &&
           (long long)((p.nx + 31) / 32) * ((p.ny + 7) / 8) < (1LL << 31) &&
           (p.nz + 7) / 8 < 65536;
}

int fused_planes(long long cols, int nz, int sms)
{
    // A CTA that marches over lz planes reads lz + 2 planes of populations
    // (the planes below and above its chunk feed its first and last
    // collisions), and the CTAs of one launch run in waves of two per SM.
    // Among equal-length chunkings with lz in [8, 64] (fewer when nz < 8),
    // take the one with the fewest waves x (lz + 2); lz = 64 stays unless
    // another length is at least 5 % cheaper (large lattices, where the last
    // wave is a small part of the launch).
    const long long slots = 2LL * (sms > 0 ? sms : 1);
    auto cost = [&](int lz) {
        const long long ctas = cols * ((nz + lz - 1) / lz);
        return ((ctas + slots - 1) / slots) * (long long)(lz + 2);
    };
    int best = nz < kPlanesMax ? nz : kPlanesMax;
    const long long c64 = cost(best);
    if (c64 > 16LL * (best + 2)) return best;   // more than 16 waves: the last one costs < 6 %
    long long cbest = c64;
    for (int nch = (nz + kPlanesMax - 1) / kPlanesMax; nch <= nz; ++nch) {
        const int lz = (nz + nch - 1) / nch;
        if (lz < kPlanesMin && nch > 1) break;
        const long long c = cost(lz);
        if (c < cbest) { cbest = c; best = lz; }
    }
    return cbest * 20 <= c64 * 19 ? best : (nz < kPlanesMax ? nz : kPlanesMax);
}

cudaError_t launch_step_fused(const HostPhys &p, const void *f_in, void *f_out, cudaStream_t s, cudaEvent_t *ev,
                              void *s_out)
{
    switch (p.storage) {
    case ST_F32: return fused::fused_t<ST_F32>(p, f_in, f_out, s, ev, s_out);
    case ST_F16_DEV: return fused::fused_t<ST_F16_DEV>(p, f_in, f_out, s, ev, s_out);
    case ST_BF16_DEV: return fused::fused_t<ST_BF16_DEV>(p, f_in, f_out, s, ev, s_out);
    case ST_F16_REL: return fused::fused_t<ST_F16_REL>(p, f_in, f_out, s, ev, s_out);
    case ST_BF16_REL: return fused::fused_t<ST_BF16_REL>(p, f_in, f_out, s, ev, s_out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
