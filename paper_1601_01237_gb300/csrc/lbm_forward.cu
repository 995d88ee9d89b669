// Forward-step kernels of the two-component D3Q19 Shan-Chen LBM
// (Otomo et al., arXiv:1601.01237, Sec. 2 and Sec. 4.1), plus state set-up,
// output fields and FP64 reductions.
//
// Two-kernel design:
//   k_density : f* (pull-gathered) -> rho^a(x)                     (Eq. 4)
//   k_collide : f* (pull-gathered), rho^b stencil -> f* (next)     (Eqs. 3-7, 13, 1/2/10)
// Populations are stored post-collision at their origin cell; a cell's
// pre-collision population f_i(x, t) is gathered from x - c_i (streaming is
// the gather), or is the reversed population of x itself when x - c_i lies
// behind a half-way bounce-back wall.
//
// Staircase walls (the inclined walls of Sec. 4.2) are a mask of solid sites
// (Phys::solid): links into a solid site bounce back, solid sites hold zero
// populations, and the density pass is followed by k_wall_rho, which gives
// each solid site the density it presents to Eq. 13.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kThreads = 256;

// Kernel parameters of the two-kernel step: the lattice's Phys plus the link
// flags of a solid mask (N words, bit i set when x - c_i is a solid site;
// nullptr without a mask).
template <class R>
struct PhysF : Phys<R> {
    const unsigned *links = nullptr;
};

// Neighbourhood of one cell: offsets of x-1, x, x+1 (and likewise y, z) as
// linear cell offsets with periodic wrap.  Index k = d + 1 for neighbour x + d.
struct Nbr {
    long long cell;
    long long xo[3], yo[3], zo[3];
    bool zlo_wall, zhi_wall;   // z - 1 (resp. z + 1) is a wall site
    int z;
};

template <class R>
__device__ __forceinline__ bool decode_cell(const Phys<R> &p, long long cell, Nbr &n)
{
    if (cell >= p.N) return false;
    const long long plane = (long long)p.nx * p.ny;
    const int z = (int)(cell / plane);
    const long long rem = cell - (long long)z * plane;
    const int y = (int)(rem / p.nx);
    const int x = (int)(rem - (long long)y * p.nx);
    n.cell = cell;
    n.z = z;
    n.xo[0] = (x == 0 ? p.nx - 1 : x - 1);
    n.xo[1] = x;
    n.xo[2] = (x == p.nx - 1 ? 0 : x + 1);
    n.yo[0] = (long long)(y == 0 ? p.ny - 1 : y - 1) * p.nx;
    n.yo[1] = (long long)y * p.nx;
    n.yo[2] = (long long)(y == p.ny - 1 ? 0 : y + 1) * p.nx;
    n.zo[0] = (long long)(z == 0 ? p.nz - 1 : z - 1) * plane;
    n.zo[1] = (long long)z * plane;
    n.zo[2] = (long long)(z == p.nz - 1 ? 0 : z + 1) * plane;
    n.zlo_wall = p.wall_z && z == 0;
    n.zhi_wall = p.wall_z && z == p.nz - 1;
    return true;
}

// Pre-collision populations of both components at one cell (streaming as a
// gather, with half-way bounce-back at z walls).
template <int S>
__device__ __forceinline__ void gather(const typename Store<S>::T *__restrict__ f,
                                       const PhysF<typename Store<S>::R> &p, const Nbr &n,
                                       typename Store<S>::R (&fa)[2][Q])
{
    using R = typename Store<S>::R;
    const unsigned lf = p.links ? __ldg(p.links + n.cell) : 0u;   // bit i: x - c_i is solid
    // reference densities of the cell (the *_REL formats code every population
    // a cell gathers relative to the cell's own stored pair; rho0 otherwise)
    R ra = p.rho0, rb = p.rho0;
    if constexpr (Store<S>::kRel) {
        const float2 rr = state_ref(f, p.ref_off)[n.cell];
        ra = rr.x; rb = rr.y;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const long long src = n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        const bool wall = (cz(i) == 1 && n.zlo_wall) || (cz(i) == -1 && n.zhi_wall) || ((lf >> i) & 1u);
        const long long idx = wall ? pair_index(opp(i), n.cell, p.N) : pair_index(i, src, p.N);
        Store<S>::load2(f + idx, w<R>(i) * ra, w<R>(i) * rb, fa[0][i], fa[1][i]);
    }
}

// Interaction sum of Eqs. 7 and 13 for both density fields at one cell:
//   S^b = sum_{i != 0} w_i c_i rho^b(x + c_i),
// where a wall site contributes rho'_b = rho_b(mirror) + rho_s^b (modified
// model) or rho_s^b (point-wise potential).  The mirror of a wall site
// x + c_i across the z wall is x + c_i with its z component replaced by z.
// The sum runs over opposite neighbours, sum_{i odd} w_i c_i (r_i - r_opp(i)),
// so that the differences of nearby densities are taken first.
template <class R>
__device__ __forceinline__ void interaction_sums(const R *__restrict__ rho, const Phys<R> &p,
                                                 const Nbr &n, R (&S)[2][3])
{
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        R sx = 0, sy = 0, sz = 0;
        const R *rb = rho + (long long)b * p.N;
        R r[Q];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && n.zlo_wall) || (cz(i) == 1 && n.zhi_wall);
            if (wall) {
                r[i] = p.rho_s[b];
                if (p.wall_mirror) r[i] += __ldg(rb + n.zo[1] + n.yo[1 + cy(i)] + n.xo[1 + cx(i)]);
            } else {
                r[i] = __ldg(rb + n.zo[1 + cz(i)] + n.yo[1 + cy(i)] + n.xo[1 + cx(i)]);
            }
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const R wr = w<R>(i) * (r[i] - r[i + 1]);
            if (cx(i) == 1) sx += wr; else if (cx(i) == -1) sx -= wr;
            if (cy(i) == 1) sy += wr; else if (cy(i) == -1) sy -= wr;
            if (cz(i) == 1) sz += wr; else if (cz(i) == -1) sz -= wr;
        }
        S[b][0] = sx; S[b][1] = sy; S[b][2] = sz;
    }
}

// Densities of both components and the mixture velocity (Eqs. 4-6); the
// momentum is summed over opposite pairs, sum_{i odd} c_i (t_i - t_opp(i)),
// t_i = f^1_i + f^2_i (the differences of nearly equal populations first).
template <class R>
__device__ __forceinline__ void local_moments(const R (&fa)[2][Q], R &r1, R &r2, R &ux, R &uy, R &uz)
{
    R rr[2], jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        R s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += fa[a][i];
        rr[a] = s;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const R v = (fa[0][i] + fa[1][i]) - (fa[0][i + 1] + fa[1][i + 1]);
        if (cx(i) == 1) jx += v; else if (cx(i) == -1) jx -= v;
        if (cy(i) == 1) jy += v; else if (cy(i) == -1) jy -= v;
        if (cz(i) == 1) jz += v; else if (cz(i) == -1) jz -= v;
    }
    r1 = rr[0];
    r2 = rr[1];
    const R inv = R(1) / (r1 + r2);
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
}

// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(kThreads)
k_density(const typename Store<S>::T *__restrict__ f, typename Store<S>::R *__restrict__ rho,
          PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    if (p.solid && p.solid[n.cell]) return;   // k_wall_rho writes solid sites
    R fa[2][Q];
    gather<S>(f, p, n, fa);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        R s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += fa[a][i];
        rho[(long long)a * p.N + n.cell] = s;
    }
}

// Density that a solid site of the mask presents to the interaction sum of
// Eq. 13, written into rho after the density pass: the modified model takes
// the mean of rho^b over the site's fluid neighbours weighted by w_i (zero
// normal derivative for fields that vary along the wall normal) plus rho_s^b;
// the original model takes rho_s^b.  A site with no fluid neighbour is never
// read by a fluid cell and gets rho_s^b.
template <class R>
__global__ void __launch_bounds__(kThreads)
k_wall_rho(R *__restrict__ rho, PhysF<R> p)
{
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    if (!p.solid[n.cell]) return;
    R num1 = 0, num2 = 0;
    int den36 = 0;   // sum of w_i over fluid neighbours, in units of 1/36
    if (p.wall_mirror) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const long long nb = n.zo[1 + cz(i)] + n.yo[1 + cy(i)] + n.xo[1 + cx(i)];
            if (__ldg(p.solid + nb)) continue;
            const R k = R(k36(i));
            num1 += k * rho[nb];
            num2 += k * rho[p.N + nb];
            den36 += k36(i);
        }
    }
    rho[n.cell] = (den36 ? num1 / R(den36) : R(0)) + p.rho_s[0];
    rho[p.N + n.cell] = (den36 ? num2 / R(den36) : R(0)) + p.rho_s[1];
}

// Link flags of a mask: bit i of cell x set when x - c_i is a solid site (so
// bit 0, x - c_0 = x, marks a solid site itself), so that the gather tests
// one word per cell instead of one byte per link.
__global__ void __launch_bounds__(kThreads)
k_link_flags(const unsigned char *__restrict__ solid, unsigned *__restrict__ links, PhysF<float> p)
{
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    unsigned f = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (solid[n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)]]) f |= 1u << i;
    links[n.cell] = f;
}

// Mask set-up of the fused step: wall_rho = rho_s at solid sites, and the
// boundary cells of the mirror model counted (lists == nullptr) or listed
// (positions from the counters; the order of a list does not matter, every
// entry is processed on its own).
__global__ void __launch_bounds__(kThreads)
k_mask_setup(const unsigned char *__restrict__ solid, const unsigned *__restrict__ links, PhysF<float> p,
             float2 *__restrict__ wall_rho, unsigned *__restrict__ bfluid, unsigned *__restrict__ bsolid,
             unsigned long long *__restrict__ counts)
{
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    const unsigned lf = links[n.cell];
    if (!(lf & 1u)) {
        if (lf) {   // a fluid cell with a solid neighbour
            const unsigned long long k = atomicAdd(counts, 1ull);
            if (bfluid) bfluid[k] = (unsigned)n.cell;
        }
        return;
    }
    wall_rho[n.cell] = make_float2(p.rho_s[0], p.rho_s[1]);
    bool fluid_nb = false;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (!solid[n.zo[1 + cz(i)] + n.yo[1 + cy(i)] + n.xo[1 + cx(i)]]) fluid_nb = true;
    if (fluid_nb) {
        const unsigned long long k = atomicAdd(counts + 1, 1ull);
        if (bsolid) bsolid[k] = (unsigned)n.cell;
    }
}

template <int S, int REG, int FORCE>
__global__ void __launch_bounds__(kThreads)
k_collide(const typename Store<S>::T *__restrict__ fin, typename Store<S>::T *__restrict__ fout,
          const typename Store<S>::R *__restrict__ rho, PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    if (p.solid && p.solid[n.cell]) {   // solid sites hold no populations
        const R e = Store<S>::kRel ? R(1) : p.rho0;   // (never read: any finite code)
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::store2(fout + pair_index(i, n.cell, p.N), R(0), R(0), w<R>(i) * e, w<R>(i) * e);
        if constexpr (Store<S>::kRel) state_ref(fout, p.ref_off)[n.cell] = make_float2(1.0f, 1.0f);
        return;
    }
    R fa[2][Q];
    gather<S>(fin, p, n, fa);
    R r1, r2, ux, uy, uz;
    local_moments(fa, r1, r2, ux, uy, uz);
    R Sb[2][3];
    interaction_sums(rho, p, n, Sb);
    // g^a = sum_b F^{ab} / rho^a + g_ext with F^{ab} = G^{ab} rho^a S^b (G^{aa} = 0)
    const R g1x = p.G12 * Sb[1][0] + p.gext[0], g1y = p.G12 * Sb[1][1] + p.gext[1],
            g1z = p.G12 * Sb[1][2] + p.gext[2];
    const R g2x = p.G21 * Sb[0][0] + p.gext[0], g2y = p.G21 * Sb[0][1] + p.gext[1],
            g2z = p.G21 * Sb[0][2] + p.gext[2];
    if (FORCE == FORCE_GUO) {   // common equilibrium velocity u* = u + g/2 (Eqs. 8-9)
        const R hi = R(0.5) / (r1 + r2);
        ux += (r1 * g1x + r2 * g2x) * hi;
        uy += (r1 * g1y + r2 * g2y) * hi;
        uz += (r1 * g1z + r2 * g2z) * hi;
    }
    collide<R, REG, FORCE>(fa[0], r1, ux, uy, uz, g1x, g1y, g1z, p.omega[0]);
    collide<R, REG, FORCE>(fa[1], r2, ux, uy, uz, g2x, g2y, g2z, p.omega[1]);
    if constexpr (Store<S>::kRel) {
        // each population coded relative to the density of the cell that reads
        // it next (x + c_i, or x itself across a wall); the cell's own pair is
        // its reference for the next gather
        const unsigned lf = p.links ? __ldg(p.links + n.cell) : 0u;
        const R d1 = rho[n.cell], d2 = rho[p.N + n.cell];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && n.zlo_wall) || (cz(i) == 1 && n.zhi_wall) ||
                              (i != 0 && ((lf >> opp(i)) & 1u));
            const long long dst = n.zo[1 + cz(i)] + n.yo[1 + cy(i)] + n.xo[1 + cx(i)];
            const R e1 = wall || i == 0 ? d1 : rho[dst], e2 = wall || i == 0 ? d2 : rho[p.N + dst];
            Store<S>::store2(fout + pair_index(i, n.cell, p.N), fa[0][i], fa[1][i], Store<S>::enc(w<R>(i) * e1),
                             Store<S>::enc(w<R>(i) * e2));
        }
        state_ref(fout, p.ref_off)[n.cell] = make_float2(d1, d2);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            Store<S>::store2(fout + pair_index(i, n.cell, p.N), fa[0][i], fa[1][i], w<R>(i) * p.rho0, w<R>(i) * p.rho0);
    }
}

// Rest-state values of one cell, formed once per cell in FP64 and rounded to
// the arithmetic type: rho^a w for the three weight classes (w = 1/3, 1/18,
// 1/36) and rho^a itself, at slot (2 q + a) N + c (q = 0, 1, 2, 3).  The
// initial populations at rest gather these instead of forming 38 FP64
// products per cell, each repeated by up to seven readers (the FP64 pipe is
// a small fraction of the FP32 one on this GPU); the values are the same
// roundings of the same FP64 products.
template <class R>
__global__ void __launch_bounds__(kThreads)
k_rest_values(const double *__restrict__ rho1, const double *__restrict__ rho2, R *__restrict__ out, long long N)
{
    const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (c >= N) return;
    const double r[2] = {rho1[c], rho2[c]};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        out[(0 + a) * N + c] = (R)(r[a] * wd(0));
        out[(2 + a) * N + c] = (R)(r[a] * wd(1));
        out[(4 + a) * N + c] = (R)(r[a] * wd(7));
        out[(6 + a) * N + c] = (R)r[a];
    }
}

// Stored value s_j(y): the population that the gather of step 0 reads as
// f_j(y + c_j), or, when y + c_j is a wall site, as f_opp(j)(y).  rest: the
// values of k_rest_values (the state at rest, u == NULL), or NULL.
template <int S>
__global__ void __launch_bounds__(kThreads)
k_init_feq(const double *__restrict__ rho1, const double *__restrict__ rho2,
           const double *__restrict__ u, const typename Store<S>::R *__restrict__ rest,
           typename Store<S>::T *__restrict__ f, PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    const bool here_solid = p.solid && p.solid[n.cell];
    const long long N = p.N;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const long long dst = n.zo[1 + cz(j)] + n.yo[1 + cy(j)] + n.xo[1 + cx(j)];
        const bool wall = (cz(j) == -1 && n.zlo_wall) || (cz(j) == 1 && n.zhi_wall) ||
                          (j != 0 && p.solid && p.solid[dst]);
        const long long src = wall ? n.cell : dst;
        const int k = wall ? opp(j) : j;
        R v1, v2, e1 = R(1), e2 = R(1);
        if (rest) {
            const int q = k == 0 ? 0 : (k < 7 ? 1 : 2);
            v1 = rest[(2 * q + 0) * N + src];
            v2 = rest[(2 * q + 1) * N + src];
            if constexpr (Store<S>::kRel) { e1 = rest[6 * N + src]; e2 = rest[7 * N + src]; }
        } else {
            // f^eq of Eq. 3 at (rho^a, u) of the source cell (u == NULL: at rest)
            double P = 1.0;
            if (u) {
                const double ux = u[3 * src], uy = u[3 * src + 1], uz = u[3 * src + 2];
                const double usq = ux * ux + uy * uy + uz * uz;
                const double cu = cdot<double>(k, ux, uy, uz);
                P = 1.0 - 1.5 * usq + cu * (3.0 - 4.5 * usq) + 4.5 * cu * cu * (1.0 + cu);
            }
            v1 = (R)(rho1[src] * wd(k) * P);
            v2 = (R)(rho2[src] * wd(k) * P);
            if constexpr (Store<S>::kRel) { e1 = (R)rho1[src]; e2 = (R)rho2[src]; }
        }
        if (here_solid) { v1 = v2 = R(0); e1 = e2 = R(1); }
        if constexpr (Store<S>::kRel) {   // coded relative to the reader's initial density
            Store<S>::store2(f + pair_index(j, n.cell, p.N), v1, v2, Store<S>::enc(w<R>(j) * e1),
                             Store<S>::enc(w<R>(j) * e2));
        } else {
            Store<S>::store2(f + pair_index(j, n.cell, p.N), v1, v2, w<R>(j) * p.rho0, w<R>(j) * p.rho0);
        }
    }
    if constexpr (Store<S>::kRel)
        state_ref(f, p.ref_off)[n.cell] = here_solid ? make_float2(1.0f, 1.0f)
                                                     : make_float2((float)rho1[n.cell], (float)rho2[n.cell]);
}

// Reference densities of a state set from explicit populations (the *_REL
// formats): each cell's densities sum_i f_i^a of the given populations
// (solid sites: 1, never read).
template <int S>
__global__ void __launch_bounds__(kThreads)
k_set_ref(const double *__restrict__ src, typename Store<S>::T *__restrict__ f, PhysF<typename Store<S>::R> p)
{
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    float2 r = make_float2(1.0f, 1.0f);
    if (!(p.solid && p.solid[n.cell])) {
        double a = 0, b = 0;
        for (int k = 0; k < Q; ++k) {
            a += src[(long long)k * p.N + n.cell];
            b += src[(long long)(Q + k) * p.N + n.cell];
        }
        r = make_float2((float)a, (float)b);
    }
    state_ref(f, p.ref_off)[n.cell] = r;
}

template <int S>
__global__ void __launch_bounds__(kThreads)
k_set_pop(const double *__restrict__ src, typename Store<S>::T *__restrict__ f,
          PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    const bool here_solid = p.solid && p.solid[n.cell];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const long long dst = n.zo[1 + cz(j)] + n.yo[1 + cy(j)] + n.xo[1 + cx(j)];
            const bool wall = (cz(j) == -1 && n.zlo_wall) || (cz(j) == 1 && n.zhi_wall) ||
                              (j != 0 && p.solid && p.solid[dst]);
            const long long sc = wall ? n.cell : dst;
            const int k = wall ? opp(j) : j;
            R e = p.rho0;   // *_REL: the reader's reference (written by k_set_ref)
            if constexpr (Store<S>::kRel) {
                const float2 rr = state_ref(f, p.ref_off)[sc];
                e = here_solid ? R(1) : (a == 0 ? rr.x : rr.y);
            }
            Store<S>::store(f + pair_index(j, n.cell, p.N) + a,
                            here_solid ? R(0) : (R)src[(long long)(a * Q + k) * p.N + sc], Store<S>::enc(w<R>(j) * e));
        }
}

template <int S>
__global__ void __launch_bounds__(kThreads)
k_get_pop(const typename Store<S>::T *__restrict__ f, double *__restrict__ dst,
          PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    const bool here_solid = p.solid && p.solid[n.cell];
    R fa[2][Q];
    gather<S>(f, p, n, fa);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i) dst[(long long)(a * Q + i) * p.N + n.cell] = here_solid ? 0.0 : (double)fa[a][i];
}

// Velocity of Eq. 8: u_F = u + g/2 with g = sum_a g^a rho^a / rho (Eq. 9).
template <class R>
__device__ __forceinline__ void velocity_uF(const Phys<R> &p, R r1, R r2, R ux, R uy, R uz,
                                            const R (&Sb)[2][3], R &fx, R &fy, R &fz)
{
    const R g1[3] = {p.G12 * Sb[1][0] + p.gext[0], p.G12 * Sb[1][1] + p.gext[1], p.G12 * Sb[1][2] + p.gext[2]};
    const R g2[3] = {p.G21 * Sb[0][0] + p.gext[0], p.G21 * Sb[0][1] + p.gext[1], p.G21 * Sb[0][2] + p.gext[2]};
    const R half_inv = R(0.5) / (r1 + r2);
    fx = ux + (g1[0] * r1 + g2[0] * r2) * half_inv;
    fy = uy + (g1[1] * r1 + g2[1] * r2) * half_inv;
    fz = uz + (g1[2] * r1 + g2[2] * r2) * half_inv;
}

template <int S, class O>
__global__ void __launch_bounds__(kThreads)
k_moments(const typename Store<S>::T *__restrict__ f, const typename Store<S>::R *__restrict__ rho,
          O *__restrict__ o1, O *__restrict__ o2, O *__restrict__ ouF, PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    Nbr n;
    if (!decode_cell(p, (long long)blockIdx.x * kThreads + threadIdx.x, n)) return;
    if (p.solid && p.solid[n.cell]) {   // no fluid at a solid site
        if (o1) o1[n.cell] = (O)0;
        if (o2) o2[n.cell] = (O)0;
        if (ouF) { ouF[3 * n.cell] = (O)0; ouF[3 * n.cell + 1] = (O)0; ouF[3 * n.cell + 2] = (O)0; }
        return;
    }
    R fa[2][Q];
    gather<S>(f, p, n, fa);
    R r1, r2, ux, uy, uz;
    local_moments(fa, r1, r2, ux, uy, uz);
    if (o1) o1[n.cell] = (O)r1;
    if (o2) o2[n.cell] = (O)r2;
    if (ouF) {
        R Sb[2][3];
        interaction_sums(rho, p, n, Sb);
        R fx, fy, fz;
        velocity_uF(p, r1, r2, ux, uy, uz, Sb, fx, fy, fz);
        ouF[3 * n.cell] = (O)fx;
        ouF[3 * n.cell + 1] = (O)fy;
        ouF[3 * n.cell + 2] = (O)fz;
    }
}

constexpr int kReduceBlocks = 1216;   // 152 SMs x 8

template <int S>
__global__ void __launch_bounds__(kThreads, 2)
k_reduce(const typename Store<S>::T *__restrict__ f, const typename Store<S>::R *__restrict__ rho,
         double *__restrict__ partials, PhysF<typename Store<S>::R> p)
{
    using R = typename Store<S>::R;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double bad = 0;
    for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < p.N;
         c += (long long)gridDim.x * kThreads) {
        Nbr n;
        decode_cell(p, c, n);
        if (p.solid && p.solid[c]) continue;   // solid sites hold no fluid
        R fa[2][Q];
        gather<S>(f, p, n, fa);
        R r1, r2, ux, uy, uz;
        local_moments(fa, r1, r2, ux, uy, uz);
        R Sb[2][3];
        interaction_sums(rho, p, n, Sb);
        R fx, fy, fz;
        velocity_uF(p, r1, r2, ux, uy, uz, Sb, fx, fy, fz);
        const double rho_t = (double)r1 + (double)r2;
        if (!(r1 > R(0)) || !(r2 > R(0)) || !isfinite((double)r1) || !isfinite((double)r2)) bad += 1;
        acc[0] += (double)r1;
        acc[1] += (double)r2;
        acc[2] += rho_t * (double)fx;
        acc[3] += rho_t * (double)fy;
        acc[4] += rho_t * (double)fz;
        // max |u_F|^2; the host takes the square root of the maximum, which
        // equals the maximum of the (correctly rounded, monotonic) roots
        acc[5] = fmax(acc[5], (double)fx * fx + (double)fy * fy + (double)fz * fz);
    }
    // fixed-order block reduction (deterministic)
    __shared__ double sh[7][kThreads];
    for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = acc[k];
    sh[6][threadIdx.x] = bad;
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            for (int k = 0; k < 7; ++k) {
                if (k == 5)
                    sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + stride]);
                else
                    sh[k][threadIdx.x] += sh[k][threadIdx.x + stride];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) partials[(long long)blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
    if (threadIdx.x == 7) partials[(long long)blockIdx.x * 8 + 7] = 0.0;
}

template <class R>
PhysF<R> make_phys(const HostPhys &h)
{
    PhysF<R> p;
    p.nx = h.nx; p.ny = h.ny; p.nz = h.nz; p.N = h.N;
    p.wall_z = h.wall_z;
    p.wall_mirror = h.wall_mirror;
    p.omega[0] = (R)(1.0 / h.tau[0]);
    p.omega[1] = (R)(1.0 / h.tau[1]);
    p.G12 = (R)h.G12; p.G21 = (R)h.G21;
    for (int d = 0; d < 3; ++d) p.gext[d] = (R)h.gext[d];
    p.rho_s[0] = (R)h.rho_s[0]; p.rho_s[1] = (R)h.rho_s[1];
    p.rho0 = (R)h.rho0;
    p.solid = h.solid;
    p.links = h.links;
    p.ref_off = h.ref_off;
    return p;
}

inline unsigned grid_for(long long N) { return (unsigned)((N + kThreads - 1) / kThreads); }

// Density pass: rho^a of every fluid cell, then (with a mask) the densities
// the solid sites present to Eq. 13.
template <int S>
void density_pass(const HostPhys &h, const typename Store<S>::T *f, typename Store<S>::R *rho, cudaStream_t s)
{
    using R = typename Store<S>::R;
    const PhysF<R> p = make_phys<R>(h);
    k_density<S><<<grid_for(h.N), kThreads, 0, s>>>(f, rho, p);
    if (h.solid) k_wall_rho<R><<<grid_for(h.N), kThreads, 0, s>>>(rho, p);
}

template <int S>
cudaError_t step_split_t(const HostPhys &h, const void *fin, void *fout, void *rho, cudaStream_t s,
                         cudaEvent_t *ev)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const PhysF<R> p = make_phys<R>(h);
    const unsigned g = grid_for(h.N);
    if (ev) cudaEventRecord(ev[0], s);
    density_pass<S>(h, (const T *)fin, (R *)rho, s);
    if (ev) cudaEventRecord(ev[1], s);
#define LBM_COLLIDE(REG_, F_) k_collide<S, REG_, F_><<<g, kThreads, 0, s>>>((const T *)fin, (T *)fout, (const R *)rho, p)
    const int reg = h.collision == LBM_REGULARIZED ? 1 : (h.collision == LBM_REGULARIZED3 ? 2 : 0);
    if (h.forcing == FORCE_GUO) {
        if (reg == 1) LBM_COLLIDE(1, FORCE_GUO); else if (reg == 2) LBM_COLLIDE(2, FORCE_GUO); else LBM_COLLIDE(0, FORCE_GUO);
    } else {
        if (reg == 1) LBM_COLLIDE(1, FORCE_EDM); else if (reg == 2) LBM_COLLIDE(2, FORCE_EDM); else LBM_COLLIDE(0, FORCE_EDM);
    }
#undef LBM_COLLIDE
    if (ev) cudaEventRecord(ev[2], s);
    return cudaGetLastError();
}

template <int S>
cudaError_t init_t(const HostPhys &h, const double *r1, const double *r2, const double *u, void *f,
                   void *scratch, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    // the eight rest values per cell fit in the other state copy
    static_assert(8 * sizeof(R) <= 2 * Q * sizeof(T), "rest values exceed a state copy");
    R *rest = nullptr;
    if (!u && scratch) {
        rest = (R *)scratch;
        k_rest_values<R><<<grid_for(h.N), kThreads, 0, s>>>(r1, r2, rest, h.N);
    }
    k_init_feq<S><<<grid_for(h.N), kThreads, 0, s>>>(r1, r2, u, rest, (T *)f, make_phys<R>(h));
    return cudaGetLastError();
}

template <int S>
cudaError_t setpop_t(const HostPhys &h, const double *src, void *f, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    if constexpr (Store<S>::kRel) k_set_ref<S><<<grid_for(h.N), kThreads, 0, s>>>(src, (T *)f, make_phys<R>(h));
    k_set_pop<S><<<grid_for(h.N), kThreads, 0, s>>>(src, (T *)f, make_phys<R>(h));
    return cudaGetLastError();
}

template <int S>
cudaError_t getpop_t(const HostPhys &h, const void *f, double *dst, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    k_get_pop<S><<<grid_for(h.N), kThreads, 0, s>>>((const T *)f, dst, make_phys<R>(h));
    return cudaGetLastError();
}

template <int S>
cudaError_t moments_t(const HostPhys &h, const void *f, void *rho, int out_f64, void *o1, void *o2,
                      void *ouF, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const PhysF<R> p = make_phys<R>(h);
    const unsigned g = grid_for(h.N);
    if (ouF) density_pass<S>(h, (const T *)f, (R *)rho, s);
    if (out_f64)
        k_moments<S, double><<<g, kThreads, 0, s>>>((const T *)f, (const R *)rho, (double *)o1,
                                                    (double *)o2, (double *)ouF, p);
    else
        k_moments<S, float><<<g, kThreads, 0, s>>>((const T *)f, (const R *)rho, (float *)o1,
                                                   (float *)o2, (float *)ouF, p);
    return cudaGetLastError();
}

template <int S>
cudaError_t reduce_t(const HostPhys &h, const void *f, void *rho, double *partials, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const PhysF<R> p = make_phys<R>(h);
    density_pass<S>(h, (const T *)f, (R *)rho, s);
    k_reduce<S><<<kReduceBlocks, kThreads, 0, s>>>((const T *)f, (const R *)rho, partials, p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_split(const HostPhys &p, const void *f_in, void *f_out, void *rho, cudaStream_t s,
                              cudaEvent_t *ev)
{
    switch (p.storage) {
    case ST_F64: return step_split_t<ST_F64>(p, f_in, f_out, rho, s, ev);
    case ST_F32: return step_split_t<ST_F32>(p, f_in, f_out, rho, s, ev);
    case ST_F16_DEV: return step_split_t<ST_F16_DEV>(p, f_in, f_out, rho, s, ev);
    case ST_BF16_DEV: return step_split_t<ST_BF16_DEV>(p, f_in, f_out, rho, s, ev);
    case ST_F16_REL: return step_split_t<ST_F16_REL>(p, f_in, f_out, rho, s, ev);
    case ST_BF16_REL: return step_split_t<ST_BF16_REL>(p, f_in, f_out, rho, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_feq(const HostPhys &p, const double *r1, const double *r2, const double *u,
                            void *f, void *scratch, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return init_t<ST_F64>(p, r1, r2, u, f, scratch, s);
    case ST_F32: return init_t<ST_F32>(p, r1, r2, u, f, scratch, s);
    case ST_F16_DEV: return init_t<ST_F16_DEV>(p, r1, r2, u, f, scratch, s);
    case ST_BF16_DEV: return init_t<ST_BF16_DEV>(p, r1, r2, u, f, scratch, s);
    case ST_F16_REL: return init_t<ST_F16_REL>(p, r1, r2, u, f, scratch, s);
    case ST_BF16_REL: return init_t<ST_BF16_REL>(p, r1, r2, u, f, scratch, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_set_populations(const HostPhys &p, const double *src, void *f, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return setpop_t<ST_F64>(p, src, f, s);
    case ST_F32: return setpop_t<ST_F32>(p, src, f, s);
    case ST_F16_DEV: return setpop_t<ST_F16_DEV>(p, src, f, s);
    case ST_BF16_DEV: return setpop_t<ST_BF16_DEV>(p, src, f, s);
    case ST_F16_REL: return setpop_t<ST_F16_REL>(p, src, f, s);
    case ST_BF16_REL: return setpop_t<ST_BF16_REL>(p, src, f, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_get_populations(const HostPhys &p, const void *f, double *dst, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return getpop_t<ST_F64>(p, f, dst, s);
    case ST_F32: return getpop_t<ST_F32>(p, f, dst, s);
    case ST_F16_DEV: return getpop_t<ST_F16_DEV>(p, f, dst, s);
    case ST_BF16_DEV: return getpop_t<ST_BF16_DEV>(p, f, dst, s);
    case ST_F16_REL: return getpop_t<ST_F16_REL>(p, f, dst, s);
    case ST_BF16_REL: return getpop_t<ST_BF16_REL>(p, f, dst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_moments(const HostPhys &p, const void *f, void *rho, int out_f64, void *o1, void *o2,
                           void *ouF, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return moments_t<ST_F64>(p, f, rho, out_f64, o1, o2, ouF, s);
    case ST_F32: return moments_t<ST_F32>(p, f, rho, out_f64, o1, o2, ouF, s);
    case ST_F16_DEV: return moments_t<ST_F16_DEV>(p, f, rho, out_f64, o1, o2, ouF, s);
    case ST_BF16_DEV: return moments_t<ST_BF16_DEV>(p, f, rho, out_f64, o1, o2, ouF, s);
    case ST_F16_REL: return moments_t<ST_F16_REL>(p, f, rho, out_f64, o1, o2, ouF, s);
    case ST_BF16_REL: return moments_t<ST_BF16_REL>(p, f, rho, out_f64, o1, o2, ouF, s);
    default: return cudaErrorInvalidValue;
    }
}

int reduce_blocks() { return kReduceBlocks; }

cudaError_t launch_mask_setup(const HostPhys &h, const unsigned char *solid, float *wall_rho, unsigned *bfluid,
                              unsigned *bsolid, unsigned long long *counts, cudaStream_t s)
{
    k_mask_setup<<<grid_for(h.N), kThreads, 0, s>>>(solid, h.links, make_phys<float>(h), (float2 *)wall_rho, bfluid,
                                                     bsolid, counts);
    return cudaGetLastError();
}

cudaError_t launch_link_flags(const HostPhys &h, const unsigned char *solid, unsigned *links, cudaStream_t s)
{
    k_link_flags<<<grid_for(h.N), kThreads, 0, s>>>(solid, links, make_phys<float>(h));
    return cudaGetLastError();
}

cudaError_t launch_density(const HostPhys &h, const void *f, void *rho, cudaStream_t s)
{
    switch (h.storage) {
    case ST_F64: density_pass<ST_F64>(h, (const double *)f, (double *)rho, s); break;
    case ST_F32: density_pass<ST_F32>(h, (const float *)f, (float *)rho, s); break;
    case ST_F16_DEV: density_pass<ST_F16_DEV>(h, (const __half *)f, (float *)rho, s); break;
    case ST_BF16_DEV: density_pass<ST_BF16_DEV>(h, (const __nv_bfloat16 *)f, (float *)rho, s); break;
    case ST_F16_REL: density_pass<ST_F16_REL>(h, (const __half *)f, (float *)rho, s); break;
    case ST_BF16_REL: density_pass<ST_BF16_REL>(h, (const __nv_bfloat16 *)f, (float *)rho, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const HostPhys &p, const void *f, void *rho, double *partials, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return reduce_t<ST_F64>(p, f, rho, partials, s);
    case ST_F32: return reduce_t<ST_F32>(p, f, rho, partials, s);
    case ST_F16_DEV: return reduce_t<ST_F16_DEV>(p, f, rho, partials, s);
    case ST_BF16_DEV: return reduce_t<ST_BF16_DEV>(p, f, rho, partials, s);
    case ST_F16_REL: return reduce_t<ST_F16_REL>(p, f, rho, partials, s);
    case ST_BF16_REL: return reduce_t<ST_BF16_REL>(p, f, rho, partials, s);
    default: return cudaErrorInvalidValue;
    }
}

size_t storage_bytes(int storage)
{
    switch (storage) {
    case ST_F64: return 8;
    case ST_F32: return 4;
    default: return 2;
    }
}

bool storage_is_rel(int storage) { return storage == ST_F16_REL || storage == ST_BF16_REL; }

size_t ref_offset(int storage, long long N)
{
    if (!storage_is_rel(storage)) return 0;
    const size_t pop = (size_t)2 * Q * (size_t)N * storage_bytes(storage);
    return (pop + 255) / 256 * 256;
}

size_t state_bytes(int storage, long long N)
{
    const size_t pop = (size_t)2 * Q * (size_t)N * storage_bytes(storage);
    return storage_is_rel(storage) ? ref_offset(storage, N) + sizeof(float) * 2 * (size_t)N : pop;
}

size_t real_bytes(int storage) { return storage == ST_F64 ? 8 : 4; }

namespace {
constexpr int kMaxSmDevices = 64;
std::atomic<int> g_device_sms[kMaxSmDevices];   // 0 = not looked up yet
}  // namespace

int current_device_sms()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= kMaxSmDevices) {   // beyond the table: look it up every time
        int n = 0;
        return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
    }
    int n = g_device_sms[dev].load(std::memory_order_acquire);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    g_device_sms[dev].store(n, std::memory_order_release);
    return n;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the two-kernel step.  Its density scratch is a
// file-scope device array (2 components x kNoallocMaxCells x 8 bytes = 32 MiB),
// present on every device that loads the library.  Host code cannot use the
// array's name as a device address, so the address is looked up once per
// device with cudaGetSymbolAddress while that device is current.
static __device__ __align__(256) unsigned char g_noalloc_rho[2 * kNoallocMaxCells * sizeof(double)];

namespace {

constexpr int kMaxDevices = 64;
void *g_noalloc_ptr[kMaxDevices] = {};

cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *ptr = __atomic_load_n(&g_noalloc_ptr[dev], __ATOMIC_ACQUIRE);
    if (!ptr) {
        e = cudaGetSymbolAddress(&ptr, g_noalloc_rho);
        if (e != cudaSuccess) return e;
        __atomic_store_n(&g_noalloc_ptr[dev], ptr, __ATOMIC_RELEASE);
    }
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_step_split_noalloc(const HostPhys &p, const void *f_in, void *f_out, cudaStream_t s)
{
    if (p.N > kNoallocMaxCells) return cudaErrorInvalidValue;
    void *rho = nullptr;
    cudaError_t e = noalloc_scratch(&rho);
    if (e != cudaSuccess) return e;
    return launch_step_split(p, f_in, f_out, rho, s);
}

}  // namespace lbm
