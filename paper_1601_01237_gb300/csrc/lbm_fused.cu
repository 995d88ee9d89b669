// Fused single-pass time step of the two-component D3Q19 Shan-Chen LBM
// (Otomo et al., arXiv:1601.01237, Sec. 2, Sec. 4.1): moments (Eqs. 4-6),
// interaction force (Eqs. 7, 13), collision with forcing (Eqs. 1-3, 10-11) and
// streaming in one kernel, with no global scratch.
//
// Each CTA owns a TX x TY column tile of the xy plane and marches along z over
// a chunk of LZ planes.  The force at plane z needs rho^b at planes z-1, z, z+1
// over the tile plus a one-cell halo; those densities live in a ring of three
// shared-memory planes.  Iteration z gathers (pull streaming) the populations
// of plane z+1, sums them into rho(z+1) for the ring, and parks them in a
// shared-memory stash; then it collides plane z with the populations parked
// in the previous iteration.  Every interior population is read from HBM once; the
// halo ring re-reads the neighbouring tiles' populations, which the
// neighbouring CTAs stream at about the same time (L2 hits).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kThreadsF = kTX * kTY;
constexpr int kHalo = 2 * (kTX + 2) + 2 * kTY;   // perimeter cells of the (TX+2) x (TY+2) box
constexpr int kLZ = 64;                           // planes per CTA

__device__ __forceinline__ int wrapi(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Pull-gather the populations of cell (x, y, z) (all in range) into fa and
// return their sums rho^1, rho^2.  xo/yo hold the wrapped x-1, x, x+1 and row
// offsets of y-1, y, y+1.
template <int S>
__device__ __forceinline__ void gather_cell(const typename Store<S>::T *__restrict__ f,
                                            const Phys<typename Store<S>::R> &p, const int (&xo)[3],
                                            const long long (&yo)[3], int z,
                                            typename Store<S>::R (&fa)[2][Q])
{
    using R = typename Store<S>::R;
    const long long plane = (long long)p.nx * p.ny;
    const long long zc = (long long)z * plane;
    const long long zm = (long long)(z == 0 ? p.nz - 1 : z - 1) * plane;
    const long long zp = (long long)(z == p.nz - 1 ? 0 : z + 1) * plane;
    const bool lo_wall = p.wall_z && z == 0;
    const bool hi_wall = p.wall_z && z == p.nz - 1;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = (cz(i) == 1 && lo_wall) || (cz(i) == -1 && hi_wall);
            long long idx;
            if (wall) {
                idx = (long long)(a * Q + opp(i)) * p.N + zc + yo[1] + xo[1];
            } else {
                const long long zs = cz(i) == 1 ? zm : (cz(i) == -1 ? zp : zc);
                idx = (long long)(a * Q + i) * p.N + zs + yo[1 - cy(i)] + xo[1 - cx(i)];
            }
            fa[a][i] = Store<S>::load(f + idx, w<R>(i) * p.rho0);
        }
    }
}

template <int S>
__device__ __forceinline__ void gather_rho(const typename Store<S>::T *__restrict__ f,
                                           const Phys<typename Store<S>::R> &p, const int (&xo)[3],
                                           const long long (&yo)[3], int z, typename Store<S>::R &r1,
                                           typename Store<S>::R &r2)
{
    using R = typename Store<S>::R;
    R fa[2][Q];
    gather_cell<S>(f, p, xo, yo, z, fa);
    R s1 = 0, s2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) { s1 += fa[0][i]; s2 += fa[1][i]; }
    r1 = s1;
    r2 = s2;
}

template <class R>
struct RhoRing {
    R v[3][2][kTY + 2][kTX + 2];
};

// Fill ring slot `slot` with rho^1, rho^2 of plane zp (zp may be -1 or nz:
// a wall ghost plane under half-way walls, else wrapped periodically).  When
// `stash` is given, interior threads also park their column's 38 populations
// there ([value][thread], conflict-free) for the collision of that plane.
template <int S>
__device__ __forceinline__ void fill_plane(const typename Store<S>::T *__restrict__ f,
                                           const Phys<typename Store<S>::R> &p, RhoRing<typename Store<S>::R> &ring,
                                           int slot, int zp, int tx0, int ty0, typename Store<S>::R *stash)
{
    using R = typename Store<S>::R;
    const int tid = threadIdx.x;
    bool ghost = false;
    int zg = zp;
    if (zp < 0 || zp >= p.nz) {
        if (p.wall_z) {
            ghost = true;
            zg = zp < 0 ? 0 : p.nz - 1;   // mirror plane across the wall
        } else {
            zg = wrapi(zp, p.nz);
        }
    }
    // interior slot of this thread (wrapped coordinates)
    {
        const int lx = tid % kTX, ly = tid / kTX;
        const int gx = (tx0 + lx) % p.nx, gy = (ty0 + ly) % p.ny;
        const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
        const long long yo[3] = {(long long)(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, (long long)gy * p.nx,
                                 (long long)(gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
        R r1, r2;
        if (ghost && !p.wall_mirror) {
            r1 = p.rho_s[0];
            r2 = p.rho_s[1];
        } else {
            R fa[2][Q];
            gather_cell<S>(f, p, xo, yo, zg, fa);
            R s1 = 0, s2 = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) { s1 += fa[0][i]; s2 += fa[1][i]; }
            r1 = s1;
            r2 = s2;
            if (ghost) {
                r1 += p.rho_s[0];
                r2 += p.rho_s[1];
            } else if (stash) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int i = 0; i < Q; ++i) stash[(a * Q + i) * kThreadsF + tid] = fa[a][i];
            }
        }
        ring.v[slot][0][ly + 1][lx + 1] = r1;
        ring.v[slot][1][ly + 1][lx + 1] = r2;
    }
    // halo perimeter
    if (tid < kHalo) {
        int hx, hy;
        if (tid < kTX + 2) { hx = tid; hy = 0; }
        else if (tid < 2 * (kTX + 2)) { hx = tid - (kTX + 2); hy = kTY + 1; }
        else { const int k = tid - 2 * (kTX + 2); hx = k < kTY ? 0 : kTX + 1; hy = 1 + (k % kTY); }
        // tile-relative coordinates may run past the domain by more than one
        // cell when the domain is smaller than a tile: reduce fully.
        int gx = (tx0 - 1 + hx) % p.nx; if (gx < 0) gx += p.nx;
        int gy = (ty0 - 1 + hy) % p.ny; if (gy < 0) gy += p.ny;
        const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
        const long long yo[3] = {(long long)(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, (long long)gy * p.nx,
                                 (long long)(gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
        R r1, r2;
        if (ghost && !p.wall_mirror) {
            r1 = p.rho_s[0];
            r2 = p.rho_s[1];
        } else {
            gather_rho<S>(f, p, xo, yo, zg, r1, r2);
            if (ghost) { r1 += p.rho_s[0]; r2 += p.rho_s[1]; }
        }
        ring.v[slot][0][hy][hx] = r1;
        ring.v[slot][1][hy][hx] = r2;
    }
}

// Force, collision and store of the interior cell of this thread at plane z,
// from the populations parked in `stash`.
template <int S, bool REG>
__device__ __forceinline__ void collide_store(typename Store<S>::T *__restrict__ fout,
                                              const Phys<typename Store<S>::R> &p,
                                              const RhoRing<typename Store<S>::R> &ring, const int (&slot)[3],
                                              int z, int x, int y, const typename Store<S>::R *stash)
{
    using R = typename Store<S>::R;
    const int tid = threadIdx.x;
    const int lx = tid % kTX + 1, ly = tid / kTX + 1;
    R fa[2][Q];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i) fa[a][i] = stash[(a * Q + i) * kThreadsF + tid];
    R r[2], jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        R s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R v = fa[a][i];
            s += v;
            if (cx(i) == 1) jx += v; else if (cx(i) == -1) jx -= v;
            if (cy(i) == 1) jy += v; else if (cy(i) == -1) jy -= v;
            if (cz(i) == 1) jz += v; else if (cz(i) == -1) jz -= v;
        }
        r[a] = s;
    }
    const R inv = R(1) / (r[0] + r[1]);
    const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
    // S^b = sum_{i != 0} w_i c_i rho^b(x + c_i)  (Eq. 7; ghost planes carry Eq. 13's rho')
    R Sb[2][3];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        R sx = 0, sy = 0, sz = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const R wr = w<R>(i) * ring.v[slot[1 + cz(i)]][b][ly + cy(i)][lx + cx(i)];
            if (cx(i) == 1) sx += wr; else if (cx(i) == -1) sx -= wr;
            if (cy(i) == 1) sy += wr; else if (cy(i) == -1) sy -= wr;
            if (cz(i) == 1) sz += wr; else if (cz(i) == -1) sz -= wr;
        }
        Sb[b][0] = sx; Sb[b][1] = sy; Sb[b][2] = sz;
    }
    collide<R, REG>(fa[0], r[0], ux, uy, uz, p.G12 * Sb[1][0] + p.gext[0], p.G12 * Sb[1][1] + p.gext[1],
                    p.G12 * Sb[1][2] + p.gext[2], p.omega[0]);
    collide<R, REG>(fa[1], r[1], ux, uy, uz, p.G21 * Sb[0][0] + p.gext[0], p.G21 * Sb[0][1] + p.gext[1],
                    p.G21 * Sb[0][2] + p.gext[2], p.omega[1]);
    const long long cell = ((long long)z * p.ny + y) * p.nx + x;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Store<S>::store(fout + (long long)(a * Q + i) * p.N + cell, fa[a][i], w<R>(i) * p.rho0);
}

constexpr size_t kStashBytes = 2 * 2 * Q * kThreadsF * sizeof(float);   // two planes, FP32

template <int S, bool REG>
__global__ void __launch_bounds__(kThreadsF, 2)
k_step_fused(const typename Store<S>::T *__restrict__ fin, typename Store<S>::T *__restrict__ fout,
             Phys<typename Store<S>::R> p, int ntx)
{
    using R = typename Store<S>::R;
    static_assert(sizeof(R) == sizeof(float), "the fused step runs FP32 arithmetic");
    __shared__ RhoRing<R> ring;
    extern __shared__ float stash_mem[];
    R *stash[2] = {(R *)stash_mem, (R *)stash_mem + 2 * Q * kThreadsF};
    const int tx0 = (blockIdx.x % ntx) * kTX;
    const int ty0 = (blockIdx.x / ntx) * kTY;
    const int z0 = blockIdx.y * kLZ;
    const int z1 = min(z0 + kLZ, p.nz);
    const int x = tx0 + threadIdx.x % kTX;
    const int y = ty0 + threadIdx.x / kTX;
    const bool active = x < p.nx && y < p.ny;

    // ring slot of plane z is (z - z0 + 1) mod 3; stash slot alternates
    fill_plane<S>(fin, p, ring, 0, z0 - 1, tx0, ty0, nullptr);
    fill_plane<S>(fin, p, ring, 1, z0, tx0, ty0, stash[0]);
    int s_m = 0, s_c = 1, s_p = 2, st = 0;
    for (int z = z0; z < z1; ++z) {
        fill_plane<S>(fin, p, ring, s_p, z + 1, tx0, ty0, z + 1 < z1 ? stash[st ^ 1] : nullptr);
        __syncthreads();
        const int sl[3] = {s_m, s_c, s_p};
        if (active) collide_store<S, REG>(fout, p, ring, sl, z, x, y, stash[st]);
        __syncthreads();
        const int t = s_m;
        s_m = s_c;
        s_c = s_p;
        s_p = t;
        st ^= 1;
    }
}
template <class R>
Phys<R> make_phys_f(const HostPhys &h)
{
    Phys<R> p;
    p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.N = h.N;
    p.wall_z = h.wall_z;
    p.wall_mirror = h.wall_mirror;
    p.omega[0] = (R)(1.0 / h.tau[0]);
    p.omega[1] = (R)(1.0 / h.tau[1]);
    p.G12 = (R)h.G12; p.G21 = (R)h.G21;
    for (int d = 0; d < 3; ++d) p.gext[d] = (R)h.gext[d];
    p.rho_s[0] = (R)h.rho_s[0]; p.rho_s[1] = (R)h.rho_s[1];
    p.rho0 = (R)h.rho0;
    return p;
}

template <int S>
cudaError_t fused_t(const HostPhys &h, const void *fin, void *fout, cudaStream_t s, cudaEvent_t *ev)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const Phys<R> p = make_phys_f<R>(h);
    const int ntx = (h.nx + kTX - 1) / kTX;
    const int nty = (h.ny + kTY - 1) / kTY;
    const dim3 grid((unsigned)(ntx * nty), (unsigned)((h.nz + kLZ - 1) / kLZ));
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kStashBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_step_fused<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kStashBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (ev) cudaEventRecord(ev[0], s);
    if (h.collision == LBM_REGULARIZED)
        k_step_fused<S, true><<<grid, kThreadsF, kStashBytes, s>>>((const T *)fin, (T *)fout, p, ntx);
    else
        k_step_fused<S, false><<<grid, kThreadsF, kStashBytes, s>>>((const T *)fin, (T *)fout, p, ntx);
    if (ev) cudaEventRecord(ev[1], s);
    return cudaGetLastError();
}

}  // namespace

bool fused_supported(const HostPhys &p)
{
    return p.storage != ST_F64 &&
           (long long)((p.nx + kTX - 1) / kTX) * ((p.ny + kTY - 1) / kTY) < (1LL << 31) &&
           (p.nz + kLZ - 1) / kLZ < 65536;
}

cudaError_t launch_step_fused(const HostPhys &p, const void *f_in, void *f_out, cudaStream_t s, cudaEvent_t *ev)
{
    switch (p.storage) {
    case ST_F32: return fused_t<ST_F32>(p, f_in, f_out, s, ev);
    case ST_F16_DEV: return fused_t<ST_F16_DEV>(p, f_in, f_out, s, ev);
    case ST_BF16_DEV: return fused_t<ST_BF16_DEV>(p, f_in, f_out, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
