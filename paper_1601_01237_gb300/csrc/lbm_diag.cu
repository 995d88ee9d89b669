// FP64 diagnostics reductions over the density fields (Sec. 3 and Sec. 4.2 of
// Otomo et al., arXiv:1601.01237): the pressure jump across a droplet
// interface for Young-Laplace (Eq. 12), and droplet volume, centre of mass and
// thin-film density for the wall cases.  The densities come from the density
// pass (k_density) into the lattice's scratch; each block writes fixed-order
// FP64 partials that the host sums in order (deterministic).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kThreadsD = 256;
constexpr int kDiagBlocks = 1216;
constexpr int kSlots = 8;

template <class R>
struct Geo {
    int nx, ny, nz;
    long long N;
    int per[3];
    const unsigned char *solid;   // mask of solid sites or nullptr
};

// Does fluid cell (x, y, z) of a masked (fully periodic) lattice have a solid
// site among its 18 neighbours?
template <class R>
__device__ __forceinline__ bool next_to_solid(const Geo<R> &g, int x, int y, int z)
{
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int m = dx * dx + dy * dy + dz * dz;
                if (m == 0 || m > 2) continue;
                const int X = (x + dx + g.nx) % g.nx, Y = (y + dy + g.ny) % g.ny, Z = (z + dz + g.nz) % g.nz;
                if (g.solid[((long long)Z * g.ny + Y) * g.nx + X]) return true;
            }
    return false;
}

__device__ __forceinline__ double min_image(double d, int n, int periodic)
{
    if (!periodic) return d;
    const double L = (double)n;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&acc)[K], double *__restrict__ partials)
{
    __shared__ double sh[K][kThreadsD];
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kThreadsD / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < K) partials[(long long)blockIdx.x * kSlots + threadIdx.x] = sh[threadIdx.x][0];
}

// Pressure p = T0 rho - G12 T0 rho^1 rho^2 (bulk pressure of the Eq. 7 force
// with G12 = G21) averaged inside r < r_in and outside r > r_out of `center`
// (minimum image along periodic axes).  Partials: sum_in, n_in, sum_out, n_out.
template <class R>
__global__ void __launch_bounds__(kThreadsD)
k_pressure(const R *__restrict__ rho, Geo<R> g, double G12, double cx, double cy, double cz, double r_in,
           double r_out, double *__restrict__ partials)
{
    double acc[4] = {0, 0, 0, 0};
    const double T0 = 1.0 / 3.0;
    const long long plane = (long long)g.nx * g.ny;
    for (long long c = (long long)blockIdx.x * kThreadsD + threadIdx.x; c < g.N; c += (long long)gridDim.x * kThreadsD) {
        const int z = (int)(c / plane);
        const long long rem = c - (long long)z * plane;
        const int y = (int)(rem / g.nx);
        const int x = (int)(rem - (long long)y * g.nx);
        if (g.solid && g.solid[c]) continue;   // no fluid at a solid site
        const double dx = min_image(x - cx, g.nx, g.per[0]);
        const double dy = min_image(y - cy, g.ny, g.per[1]);
        const double dz = min_image(z - cz, g.nz, g.per[2]);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double r1 = (double)rho[c], r2 = (double)rho[g.N + c];
        const double p = T0 * (r1 + r2) - G12 * T0 * r1 * r2;
        if (r < r_in) { acc[0] += p; acc[1] += 1.0; }
        if (r > r_out) { acc[2] += p; acc[3] += 1.0; }
    }
    block_reduce_store<4>(acc, partials);
}

// Droplet of component 1: cells with rho^1 > threshold.  Partials: volume,
// sum x, sum y, sum z (coordinates relative to `origin`, minimum image along
// periodic axes), sum rho^1 over the droplet, and over the wall layer outside
// the droplet: sum rho^1 and cell count (thin film).  The wall layer is z = 0,
// or with a mask the fluid cells next to a solid site; solid sites count for
// nothing.
template <class R>
__global__ void __launch_bounds__(kThreadsD)
k_droplet(const R *__restrict__ rho, Geo<R> g, double threshold, double ox, double oy, double oz,
          double *__restrict__ partials)
{
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const long long plane = (long long)g.nx * g.ny;
    for (long long c = (long long)blockIdx.x * kThreadsD + threadIdx.x; c < g.N; c += (long long)gridDim.x * kThreadsD) {
        const int z = (int)(c / plane);
        const long long rem = c - (long long)z * plane;
        const int y = (int)(rem / g.nx);
        const int x = (int)(rem - (long long)y * g.nx);
        if (g.solid && g.solid[c]) continue;
        const double r1 = (double)rho[c];
        if (r1 > threshold) {
            acc[0] += 1.0;
            acc[1] += min_image(x - ox, g.nx, g.per[0]);
            acc[2] += min_image(y - oy, g.ny, g.per[1]);
            acc[3] += min_image(z - oz, g.nz, g.per[2]);
            acc[4] += r1;
        } else if (g.solid ? next_to_solid(g, x, y, z) : z == 0) {
            acc[5] += r1;
            acc[6] += 1.0;
        }
    }
    block_reduce_store<7>(acc, partials);
}

template <class R>
Geo<R> geo_of(const HostPhys &h)
{
    Geo<R> g;
    g.nx = h.nx; g.ny = h.ny; g.nz = h.nz; g.N = h.N;
    g.per[0] = 1; g.per[1] = 1; g.per[2] = h.wall_z ? 0 : 1;
    g.solid = h.solid;
    return g;
}

}  // namespace

int diag_blocks() { return kDiagBlocks; }
int diag_slots() { return kSlots; }

cudaError_t launch_pressure(const HostPhys &h, const void *rho, const double center[3], double r_in, double r_out,
                            double *partials, cudaStream_t s)
{
    if (h.storage == ST_F64)
        k_pressure<double><<<kDiagBlocks, kThreadsD, 0, s>>>((const double *)rho, geo_of<double>(h), h.G12, center[0],
                                                             center[1], center[2], r_in, r_out, partials);
    else
        k_pressure<float><<<kDiagBlocks, kThreadsD, 0, s>>>((const float *)rho, geo_of<float>(h), h.G12, center[0],
                                                            center[1], center[2], r_in, r_out, partials);
    return cudaGetLastError();
}

cudaError_t launch_droplet(const HostPhys &h, const void *rho, double threshold, const double origin[3],
                           double *partials, cudaStream_t s)
{
    if (h.storage == ST_F64)
        k_droplet<double><<<kDiagBlocks, kThreadsD, 0, s>>>((const double *)rho, geo_of<double>(h), threshold,
                                                            origin[0], origin[1], origin[2], partials);
    else
        k_droplet<float><<<kDiagBlocks, kThreadsD, 0, s>>>((const float *)rho, geo_of<float>(h), threshold,
                                                           origin[0], origin[1], origin[2], partials);
    return cudaGetLastError();
}

}  // namespace lbm
