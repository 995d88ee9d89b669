// Reverse-mode step of the two-component D3Q19 Shan-Chen update: dispatch
// over the storage formats (the per-format instances of the reverse step live
// in lbm_adjoint_<format>.cu), the seed of the adjoint fields and the
// initial-density gradient.  Kernels and notation: lbm_adjoint_impl.cuh.
#include "lbm_adjoint_impl.cuh"

namespace lbm {

extern template cudaError_t adj::adj_step_t<ST_F64>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
extern template cudaError_t adj::adj_step_t<ST_F32>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
extern template cudaError_t adj::adj_step_t<ST_F16_DEV>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
extern template cudaError_t adj::adj_step_t<ST_BF16_DEV>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
extern template cudaError_t adj::adj_step_t<ST_F16_REL>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);
extern template cudaError_t adj::adj_step_t<ST_BF16_REL>(const HostPhys &, const void *, const void *, int,
                                       const void *, const void *, void *, void *, void *, double *,
                                       cudaStream_t);

// One resident wave of k_adj_local on the current device for a storage
// format: AdjLaunch::blocks CTAs on every SM.
int adjoint_blocks(int storage)
{
    const int per_sm = storage == ST_F64 ? AdjLaunch<double>::blocks : AdjLaunch<float>::blocks;
    return per_sm * current_device_sms();
}

cudaError_t launch_adjoint_step(const HostPhys &p, const void *f, const void *rho, int rho_is_sums, const void *lam_next,
                                const void *Dn, void *lam_loc, void *a, void *Dout, double *partials, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return adj::adj_step_t<ST_F64>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    case ST_F32: return adj::adj_step_t<ST_F32>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    case ST_F16_DEV: return adj::adj_step_t<ST_F16_DEV>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    case ST_BF16_DEV: return adj::adj_step_t<ST_BF16_DEV>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    case ST_F16_REL: return adj::adj_step_t<ST_F16_REL>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    case ST_BF16_REL: return adj::adj_step_t<ST_BF16_REL>(p, f, rho, rho_is_sums, lam_next, Dn, lam_loc, a, Dout, partials, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_seed(const HostPhys &p, const void *g1, const void *g2, int g_f64, void *lam,
                                cudaStream_t s)
{
    if (p.storage == ST_F64) {
        if (g_f64) k_adj_seed<double, double><<<gridA(p.N), kThreadsA, 0, s>>>((const double *)g1, (const double *)g2, (double *)lam, p.N);
        else k_adj_seed<double, float><<<gridA(p.N), kThreadsA, 0, s>>>((const float *)g1, (const float *)g2, (double *)lam, p.N);
    } else {
        if (g_f64) k_adj_seed<float, double><<<gridA(p.N), kThreadsA, 0, s>>>((const double *)g1, (const double *)g2, (float *)lam, p.N);
        else k_adj_seed<float, float><<<gridA(p.N), kThreadsA, 0, s>>>((const float *)g1, (const float *)g2, (float *)lam, p.N);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rho0(const HostPhys &p, const void *lam, const void *D, double *g1, double *g2,
                                cudaStream_t s)
{
    if (p.storage == ST_F64)
        k_adj_rho0<double><<<gridA(p.N), kThreadsA, 0, s>>>((const double *)lam, (const double *)D, g1, g2, p.N,
                                                            p.solid);
    else
        k_adj_rho0<float><<<gridA(p.N), kThreadsA, 0, s>>>((const float *)lam, (const float *)D, g1, g2, p.N,
                                                           p.solid);
    return cudaGetLastError();
}

}  // namespace lbm
