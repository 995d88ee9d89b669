// Fused single-pass time step (kernel templates; instantiated per storage
// format in lbm_fused_<format>.cu) of the two-component D3Q19 Shan-Chen LBM
// (Otomo et al., arXiv:1601.01237, Sec. 2, Sec. 4.1): moments (Eqs. 4-6),
// interaction force (Eqs. 7, 13), collision with forcing (Eqs. 1-3, 10-11) and
// streaming in one kernel, with no global scratch.
//
// Each CTA owns a 32 x 8 column tile of the xy plane and marches along z over
// a chunk of 8 to 64 planes (fused_planes balances the CTA waves), one
// thread per column.
// The force at plane z needs rho^b at planes z-1, z, z+1 over the tile plus a
// one-cell halo; those densities live in a ring of four shared-memory planes.
// Iteration z:
//   A. every thread takes its column's 38 populations of plane z+1 from
//      registers (19 paired loads of both components issued one iteration
//      earlier): the (rho^1, rho^2) pair into the ring, momentum into a moment
//      buffer, the (f^1_i, f^2_i) pairs into a shared-memory stash (one 8-byte
//      shared access per pair); for the halo ring of plane z+2 it gathers 6 or
//      7 of the 19 directions of one halo cell (84 halo cells x 3 groups, both
//      components per load), summed into fixed-order partial densities; the
//      halo densities of plane z+1 (partials gathered one iteration earlier)
//      are completed in the ring.  The side-column halo cells cost one
//      scattered sector per load, so their tasks are spread evenly over the
//      warps (6 per warp) next to runs of consecutive row-halo tasks;
//   -- one barrier --
//   B. every thread issues the interior gathers of plane z+2 into registers,
//      then collides its column at plane z from its stash entries and stores
//      the post-collision populations, so that the loads are in flight
//      during the collision.
// Phase A of iteration z+1 writes only the ring slot of plane z+2, the
// thread's own stash and moment entries and the halo partials of plane z+3,
// none of which phase B of iteration z reads, so one barrier per plane
// suffices and fast warps start the next plane while slow warps finish their
// collisions.  Interior and halo loads are balanced over all threads; every
// interior population is read from HBM once and written once, and the halo
// re-reads neighbouring tiles' populations that the neighbouring CTAs stream
// at about the same time (L2 hits).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace fused {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kThreadsF = kTX * kTY;
constexpr int kHalo = 2 * (kTX + 2) + 2 * kTY;   // perimeter cells of the (TX+2) x (TY+2) box
constexpr int kGroups = 3;                        // halo directions split 7 + 6 + 6 (both components each)
constexpr int kPer = 14;
constexpr int Q2 = 2 * Q;
static_assert(kGroups * kHalo <= kThreadsF, "one halo group per thread");

template <class R>
struct FusedSmem {
    float2 ring[4][kTY + 2][kTX + 2];      // (rho^1, rho^2) of planes z-1 .. z+2 (+ halo)
    R hpart[2][kGroups][2][kHalo];         // halo partial densities of the next two planes
    R mom[2][3][kThreadsF];                // sum_a sum_i c_i f_i of the stashed planes
    float2 stash[2][Q][kThreadsF];         // pre-collision (f^1_i, f^2_i) of planes z, z+1
    unsigned char hsolid[2][kHalo];        // under a mask: the halo cell is a solid site
};

// *_REL formats: the reciprocals (1/rho^1, 1/rho^2) of the ring densities, in
// four more planes of shared memory behind FusedSmem.  A population is coded
// relative to its destination's density, and every ring density is the
// destination of up to 27 populations, so its reciprocal is formed once, where
// the ring is written.
using InvRing = float2[kTY + 2][kTX + 2];

template <int S>
constexpr size_t smem_bytes()
{
    return sizeof(FusedSmem<float>) + (Store<S>::kRel ? 4 * sizeof(InvRing) : 0);
}

// Writes one ring density pair (and, for the *_REL formats, its reciprocals).
template <int S>
__device__ __forceinline__ void put_ring(FusedSmem<typename Store<S>::R> &sm, InvRing *inv, int slot, int y, int x,
                                         float r1, float r2)
{
    sm.ring[slot][y][x] = make_float2(r1, r2);
    if constexpr (Store<S>::kRel) inv[slot][y][x] = make_float2(__frcp_rn(r1), __frcp_rn(r2));
}

// A lattice column (x, y) with its wrapped neighbour offsets.
struct Col {
    int xo[3];   // x-1, x, x+1
    int yo[3];   // (y-1, y, y+1) * nx
};

__device__ __forceinline__ Col make_col(int gx, int gy, int nx, int ny)
{
    Col c;
    c.xo[0] = gx == 0 ? nx - 1 : gx - 1;
    c.xo[1] = gx;
    c.xo[2] = gx == nx - 1 ? 0 : gx + 1;
    c.yo[0] = (gy == 0 ? ny - 1 : gy - 1) * nx;
    c.yo[1] = gy * nx;
    c.yo[2] = (gy == ny - 1 ? 0 : gy + 1) * nx;
    return c;
}

// Plane set-up for a gather at plane zp: the plane actually read (zp wrapped,
// or the mirror plane of a wall ghost) and its z neighbour offsets.
struct PlaneRef {
    int zc, zm, zp;        // offsets of planes z, z-1, z+1 (wrapped)
    bool lo_wall, hi_wall; // half-way wall below / above plane z
    bool ghost;            // zp is a wall ghost plane (density = mirror + rho_s)
    bool constant;         // ghost plane with the point-wise wall potential: rho = rho_s
};

template <bool WALLZ, class R>
__device__ __forceinline__ PlaneRef plane_ref(const Phys<R> &p, int zp)
{
    PlaneRef r;
    int z = zp;
    r.ghost = false;
    if (zp < 0 || zp >= p.nz) {
        if (WALLZ) {
            r.ghost = true;
            z = zp < 0 ? 0 : p.nz - 1;
        } else {
            z = ((zp % p.nz) + p.nz) % p.nz;
        }
    }
    r.constant = r.ghost && !p.wall_mirror;
    const int plane = p.nx * p.ny;
    r.zc = z * plane;
    r.zm = (z == 0 ? p.nz - 1 : z - 1) * plane;
    r.zp = (z == p.nz - 1 ? 0 : z + 1) * plane;
    r.lo_wall = WALLZ && z == 0;
    r.hi_wall = WALLZ && z == p.nz - 1;
    return r;
}

// Element index (within its population array) and array number of the
// pull-gathered population i of component a at column c of plane pr.  lw is
// the cell's link word under a solid mask (bit i: x - c_i is a solid site,
// whose link bounces back), 0 without one.
template <int I>
__device__ __forceinline__ int gather_elem(const PlaneRef &pr, const Col &c, unsigned lw, int &arr_dir)
{
    const bool wall = (cz(I) == 1 && pr.lo_wall) || (cz(I) == -1 && pr.hi_wall) || (I != 0 && ((lw >> I) & 1u));
    if (wall) {
        arr_dir = opp(I);
        return pr.zc + c.yo[1] + c.xo[1];
    }
    arr_dir = I;
    const int zs = cz(I) == 1 ? pr.zm : (cz(I) == -1 ? pr.zp : pr.zc);
    return zs + c.yo[1 - cy(I)] + c.xo[1 - cx(I)];
}

// Reference densities that decode the populations gathered into column c of
// plane pr: the cell's own stored pair for the *_REL formats, rho0 otherwise.
template <int S>
__device__ __forceinline__ float2 gather_ref(const typename Store<S>::T *__restrict__ f,
                                             const Phys<typename Store<S>::R> &p, const PlaneRef &pr, const Col &c)
{
    if constexpr (Store<S>::kRel)
        return state_ref(f, p.ref_off)[(unsigned)(pr.zc + c.yo[1] + c.xo[1])];
    else
        return make_float2((float)p.rho0, (float)p.rho0);
}

// Element offsets inside one component's 19 arrays fit 32 bits (19 N < 2^32,
// checked on the host): one multiply-add per load instead of 64-bit index math.
template <int S, int I>
__device__ __forceinline__ void load_dir(const typename Store<S>::T *__restrict__ f, long long N,
                                         float2 rr, const PlaneRef &pr, const Col &c, unsigned lw,
                                         typename Store<S>::R (&v)[Q2])
{
    using R = typename Store<S>::R;
    int d;
    const int e = gather_elem<I>(pr, c, lw, d);
    const unsigned idx = (unsigned)d * (unsigned)N + (unsigned)e;
    if constexpr (Store<S>::kDev)   // the deviation formats compute in d = f - w rho0
        Store<S>::load2_d(f + 2 * (size_t)idx, v[I], v[Q + I]);
    else
        Store<S>::load2(f + 2 * (size_t)idx, w<R>(I) * rr.x, w<R>(I) * rr.y, v[I], v[Q + I]);
}

template <int S, int I>
struct GatherAll {
    __device__ __forceinline__ static void run(const typename Store<S>::T *__restrict__ f, long long N,
                                               float2 rr, const PlaneRef &pr, const Col &c, unsigned lw,
                                               typename Store<S>::R (&v)[Q2])
    {
        load_dir<S, I>(f, N, rr, pr, c, lw, v);
        GatherAll<S, I + 1>::run(f, N, rr, pr, c, lw, v);
    }
};
template <int S>
struct GatherAll<S, Q> {
    __device__ __forceinline__ static void run(const typename Store<S>::T *__restrict__, long long,
                                               float2, const PlaneRef &, const Col &, unsigned,
                                               typename Store<S>::R (&)[Q2]) {}
};

// The same gather with the pairs kept as stored (one 32-bit word per pair in
// the 16-bit formats), decoded where they are used (decode_all): a plane in
// flight across the collision then holds 19 registers instead of 38.
template <int S, int I>
struct GatherRaw {
    __device__ __forceinline__ static void run(const typename Store<S>::T *__restrict__ f, long long N,
                                               const PlaneRef &pr, const Col &c, unsigned lw,
                                               typename Store<S>::Raw (&r)[Q])
    {
        int d;
        const int e = gather_elem<I>(pr, c, lw, d);
        r[I] = Store<S>::load_raw(f + 2 * (size_t)((unsigned)d * (unsigned)N + (unsigned)e));
        GatherRaw<S, I + 1>::run(f, N, pr, c, lw, r);
    }
};
template <int S>
struct GatherRaw<S, Q> {
    __device__ __forceinline__ static void run(const typename Store<S>::T *__restrict__, long long, const PlaneRef &,
                                               const Col &, unsigned, typename Store<S>::Raw (&)[Q]) {}
};

template <int S>
__device__ __forceinline__ void decode_all(const typename Store<S>::Raw (&r)[Q], float2 rr,
                                           typename Store<S>::R (&v)[Q2])
{
    using R = typename Store<S>::R;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if constexpr (Store<S>::kDev)
            Store<S>::decode2_d(r[i], v[i], v[Q + i]);
        else
            Store<S>::decode2(r[i], w<R>(i) * rr.x, w<R>(i) * rr.y, v[i], v[Q + i]);
    }
}

// rho^1, rho^2 and momentum of a gathered population set.  The densities are
// summed in the grouping of the halo partial gathers, (directions 0-6 +
// directions 7-12) + directions 13-18, so that a cell's density is the same
// bit for bit whether its own CTA forms it or a neighbouring CTA forms it as a
// halo cell.  The momentum is summed over opposite pairs,
// sum_{i odd} c_i (t_i - t_opp(i)) with t_i = f^1_i + f^2_i: the same sum, but
// each difference of two nearly equal populations is taken first (exactly,
// in FP32, when they are within a factor of two), so the rounding of the
// result scales with the momentum, not with the density.
template <class R>
__device__ __forceinline__ void sums(const R (&v)[Q2], R &r1, R &r2, R &jx, R &jy, R &jz)
{
    R s1 = 0, s2 = 0, ax = 0, ay = 0, az = 0;
    {
        R g1[3] = {0, 0, 0}, g2[3] = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int k = i < 7 ? 0 : (i < 13 ? 1 : 2);
            g1[k] += v[i];
            g2[k] += v[Q + i];
        }
        s1 = g1[0] + g1[1] + g1[2];
        s2 = g2[0] + g2[1] + g2[2];
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const R t = (v[i] + v[Q + i]) - (v[i + 1] + v[Q + i + 1]);
        if (cx(i) == 1) ax += t; else if (cx(i) == -1) ax -= t;
        if (cy(i) == 1) ay += t; else if (cy(i) == -1) ay -= t;
        if (cz(i) == 1) az += t; else if (cz(i) == -1) az -= t;
    }
    r1 = s1; r2 = s2; jx = ax; jy = ay; jz = az;
}

// Partial gather of one halo cell: directions [D, D1) of both components
// (one paired load each), summed per component.
template <int S, int D, int D1>
struct HaloRange {
    __device__ __forceinline__ static void load(const typename Store<S>::T *__restrict__ f, long long N,
                                                float2 rr, const PlaneRef &pr, const Col &c, unsigned lw,
                                                typename Store<S>::R (&v)[kPer], int k)
    {
        using R = typename Store<S>::R;
        int d;
        const int e = gather_elem<D>(pr, c, lw, d);
        const unsigned idx = (unsigned)d * (unsigned)N + (unsigned)e;
        if constexpr (Store<S>::kDev)
            Store<S>::load2_d(f + 2 * (size_t)idx, v[k], v[k + 1]);
        else
            Store<S>::load2(f + 2 * (size_t)idx, w<R>(D) * rr.x, w<R>(D) * rr.y, v[k], v[k + 1]);
        HaloRange<S, D + 1, D1>::load(f, N, rr, pr, c, lw, v, k + 2);
    }
    __device__ __forceinline__ static void sum(const typename Store<S>::R (&v)[kPer], int k,
                                               typename Store<S>::R &s0, typename Store<S>::R &s1)
    {
        s0 += v[k];
        s1 += v[k + 1];
        HaloRange<S, D + 1, D1>::sum(v, k + 2, s0, s1);
    }
};
template <int S, int D1>
struct HaloRange<S, D1, D1> {
    __device__ __forceinline__ static void load(const typename Store<S>::T *__restrict__, long long,
                                                float2, const PlaneRef &, const Col &, unsigned,
                                                typename Store<S>::R (&)[kPer], int) {}
    __device__ __forceinline__ static void sum(const typename Store<S>::R (&)[kPer], int,
                                               typename Store<S>::R &, typename Store<S>::R &) {}
};

template <int S>
__device__ __forceinline__ void halo_load(const typename Store<S>::T *__restrict__ f, const Phys<typename Store<S>::R> &p,
                                          const PlaneRef &pr, const Col &c, unsigned lw, int g,
                                          typename Store<S>::R (&v)[kPer])
{
    const float2 rr = gather_ref<S>(f, p, pr, c);
    if (g == 0) HaloRange<S, 0, 7>::load(f, p.N, rr, pr, c, lw, v, 0);
    else if (g == 1) HaloRange<S, 7, 13>::load(f, p.N, rr, pr, c, lw, v, 0);
    else HaloRange<S, 13, Q>::load(f, p.N, rr, pr, c, lw, v, 0);
}

template <int S>
__device__ __forceinline__ void halo_sum(const typename Store<S>::R (&v)[kPer], int g, typename Store<S>::R &s0,
                                         typename Store<S>::R &s1)
{
    s0 = 0;
    s1 = 0;
    if (g == 0) HaloRange<S, 0, 7>::sum(v, 0, s0, s1);
    else if (g == 1) HaloRange<S, 7, 13>::sum(v, 0, s0, s1);
    else HaloRange<S, 13, Q>::sum(v, 0, s0, s1);
}

// Collision of both components at the thread's interior cell of plane z (the
// populations come from the stash, densities from the ring, momentum from the
// moment buffer), forcing term included, result stored at the cell.
// With the *_REL formats each stored population is coded relative to the
// density of the cell that reads it next: x + c_i (from the ring), or the
// cell itself when x + c_i lies behind a wall (lo_wall / hi_wall: plane z is
// next to the lower / upper wall); the cell's own densities are stored as the
// reference of the populations it will gather.
// Under a solid mask, lw is the cell's link word: a solid site (bit 0) stores
// zero populations (reference densities 1 for the *_REL formats) and zero
// interaction sums, and a population whose destination x + c_i is solid
// (bit opp(i)) returns to the cell itself.
template <int S, int REG, int FORCE>
__device__ __forceinline__ void collide_cell(typename Store<S>::T *__restrict__ fout, const Phys<typename Store<S>::R> &p,
                                             const FusedSmem<typename Store<S>::R> &sm, const InvRing *rinv,
                                             int sl_m, int sl_c, int sl_p,
                                             int st, long long cell, typename Store<S>::R *__restrict__ s_out,
                                             bool lo_wall, bool hi_wall, unsigned lw = 0u)
{
    using R = typename Store<S>::R;
    const int tid = threadIdx.x;
    if (lw & 1u) {   // solid site
        typename Store<S>::T *os = fout + 2 * cell;
        const unsigned n32 = (unsigned)p.N;
#pragma unroll
        for (int i = 0; i < Q && fout; ++i) {
            // zero in every format: the deviation formats code it against w_i rho0,
            // the relative ones code 0 as 0 whatever their parameter
            const R ref = Store<S>::kRel ? R(1) : w<R>(i) * R(p.rho0);
            Store<S>::store2(os + 2 * (size_t)((unsigned)i * n32), R(0), R(0), ref, ref);
        }
        if constexpr (Store<S>::kRel) {
            if (fout) state_ref(fout, p.ref_off)[cell] = make_float2(1.0f, 1.0f);
        }
        if (s_out) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s_out[(long long)k * p.N + cell] = R(0);
        }
        return;
    }
    const int lx = tid % kTX + 1, ly = tid / kTX + 1;
    const float2 rr = sm.ring[sl_c][ly][lx];
    const R r1 = rr.x, r2 = rr.y;
    const R inv = R(1) / (r1 + r2);
    R ux = sm.mom[st][0][tid] * inv, uy = sm.mom[st][1][tid] * inv, uz = sm.mom[st][2][tid] * inv;
    // S^b = sum_{i != 0} w_i c_i rho^b(x + c_i)  (Eq. 7; ghost planes carry
    // Eq. 13's rho'), summed over opposite neighbours as
    // sum_{i odd} w_i c_i (rho^b(x + c_i) - rho^b(x - c_i)): the differences of
    // nearby densities come first, so the rounding scales with the gradient
    // rather than with the density
    R Sb[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int slp = cz(i) == -1 ? sl_m : (cz(i) == 1 ? sl_p : sl_c);
        const int slm = cz(i) == -1 ? sl_p : (cz(i) == 1 ? sl_m : sl_c);
        const float2 rp = sm.ring[slp][ly + cy(i)][lx + cx(i)];
        const float2 rm = sm.ring[slm][ly - cy(i)][lx - cx(i)];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const R wr = w<R>(i) * (b == 0 ? rp.x - rm.x : rp.y - rm.y);
            if (cx(i) == 1) Sb[b][0] += wr; else if (cx(i) == -1) Sb[b][0] -= wr;
            if (cy(i) == 1) Sb[b][1] += wr; else if (cy(i) == -1) Sb[b][1] -= wr;
            if (cz(i) == 1) Sb[b][2] += wr; else if (cz(i) == -1) Sb[b][2] -= wr;
        }
    }
    if (s_out) {   // interaction sums of this step (reverse-mode replay)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d) s_out[(long long)(3 * b + d) * p.N + cell] = Sb[b][d];
    }
    if (!fout) return;   // the interaction sums alone (the last step of a replayed segment)
    // g^a = sum_b F^{ab} / rho^a + g_ext = G^{ab} S^b + g_ext
    R v1x = ux + p.G12 * Sb[1][0] + p.gext[0], v1y = uy + p.G12 * Sb[1][1] + p.gext[1],
      v1z = uz + p.G12 * Sb[1][2] + p.gext[2];
    R v2x = ux + p.G21 * Sb[0][0] + p.gext[0], v2y = uy + p.G21 * Sb[0][1] + p.gext[1],
      v2z = uz + p.G21 * Sb[0][2] + p.gext[2];
    // Guo forcing: both components relax toward f^eq(u*) with the common
    // u* = u + (F^1 + F^2) / (2 rho) (Eqs. 8-9), F^a = rho^a g^a, and gain the
    // forcing term cf (k_i / 36) (even_i +- odd_i), even = 9 (c.u*)(c.F) - 3 u*.F,
    // odd = 3 c.F, cf = 1 - 1/(2 tau) (BGK) or 1/2 (regularized); the
    // exact-difference reading's formulas below then take u = v^1 = v^2 = u*
    R F1x = 0, F1y = 0, F1z = 0, F2x = 0, F2y = 0, F2z = 0, uF1 = 0, uF2 = 0, cf1 = 0, cf2 = 0;
    if constexpr (FORCE == FORCE_GUO) {
        F1x = r1 * (v1x - ux); F1y = r1 * (v1y - uy); F1z = r1 * (v1z - uz);
        F2x = r2 * (v2x - ux); F2y = r2 * (v2y - uy); F2z = r2 * (v2z - uz);
        const R hi = R(0.5) * inv;
        ux += (F1x + F2x) * hi; uy += (F1y + F2y) * hi; uz += (F1z + F2z) * hi;
        v1x = ux; v1y = uy; v1z = uz;
        v2x = ux; v2y = uy; v2z = uz;
        uF1 = ux * F1x + uy * F1y + uz * F1z;
        uF2 = ux * F2x + uy * F2y + uz * F2z;
        cf1 = REG ? R(0.5) : R(1) - R(0.5) * p.omega[0];
        cf2 = REG ? R(0.5) : R(1) - R(0.5) * p.omega[1];
    }
    const R usq = ux * ux + uy * uy + uz * uz;
    const R v1sq = v1x * v1x + v1y * v1y + v1z * v1z;
    const R v2sq = v2x * v2x + v2y * v2y + v2z * v2z;
    const R Au = R(1) - R(1.5) * usq, Bu = R(3) - R(4.5) * usq;
    const R A1 = R(1) - R(1.5) * v1sq, B1 = R(3) - R(4.5) * v1sq;
    const R A2 = R(1) - R(1.5) * v2sq, B2 = R(3) - R(4.5) * v2sq;
    const R keep1 = R(1) - p.omega[0], keep2 = R(1) - p.omega[1];
    const float2 *s0 = &sm.stash[st][0][tid];
    const R rq1 = r1 / R(36), rq2 = r2 / R(36);   // rho w_i = (rho / 36) k_i
    typename Store<S>::T *o = fout + 2 * cell;   // (component 1, component 2) of direction 0
    const unsigned N32 = (unsigned)p.N;
    const R ref0 = p.rho0;
    // Deviation formats: the stash holds d = f - w rho0 and the outputs are
    // stored as f* - w rho0; that adds to each output a constant per unit
    // weight: -omega rho0 under BGK (keep f = keep d + keep w rho0), -rho0
    // under the regularized filter (which keeps no f of its own)
    const R dc1 = Store<S>::kDev ? (REG ? ref0 : p.omega[0] * ref0) : R(0);
    const R dc2 = Store<S>::kDev ? (REG ? ref0 : p.omega[1] * ref0) : R(0);

    // Regularized: second moments of f - f^eq(u): Pi = sum c c f - rho (T0 I + u u)
    R P1[6], P2[6], t1 = 0, t2 = 0;
    Third<R> th1, th2;   // REG = 2: third-order moments of f - f^eq(u)
    if (REG) {
#pragma unroll
        for (int k = 0; k < 6; ++k) { P1[k] = 0; P2[k] = 0; }
        if (REG == 2) { th1.zero(); th2.zero(); }
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const float2 fp = s0[i * kThreadsF];
            const R fa = fp.x, fb = fp.y;
            if (REG == 2) { th1.add(i, fa); th2.add(i, fb); }
            if (cx(i)) { P1[0] += fa; P2[0] += fb; }
            if (cy(i)) { P1[1] += fa; P2[1] += fb; }
            if (cz(i)) { P1[2] += fa; P2[2] += fb; }
            if (cx(i) && cy(i)) { if (cx(i) == cy(i)) { P1[3] += fa; P2[3] += fb; } else { P1[3] -= fa; P2[3] -= fb; } }
            if (cx(i) && cz(i)) { if (cx(i) == cz(i)) { P1[4] += fa; P2[4] += fb; } else { P1[4] -= fa; P2[4] -= fb; } }
            if (cy(i) && cz(i)) { if (cy(i) == cz(i)) { P1[5] += fa; P2[5] += fb; } else { P1[5] -= fa; P2[5] -= fb; } }
        }
        const R T0 = R(1) / R(3);
        if constexpr (Store<S>::kDev) {   // sum_i c_i c_i w_i rho0 = rho0 T0 I
            const R d = ref0 * T0;
            P1[0] += d; P1[1] += d; P1[2] += d;
            P2[0] += d; P2[1] += d; P2[2] += d;
        }
        P1[0] -= r1 * (T0 + ux * ux); P2[0] -= r2 * (T0 + ux * ux);
        P1[1] -= r1 * (T0 + uy * uy); P2[1] -= r2 * (T0 + uy * uy);
        P1[2] -= r1 * (T0 + uz * uz); P2[2] -= r2 * (T0 + uz * uz);
        P1[3] -= r1 * ux * uy; P2[3] -= r2 * ux * uy;
        if constexpr (FORCE == FORCE_GUO) {   // Pi of f - f^eq(u*) + F/2: + (u* F + F u*) / 2
            P1[0] += ux * F1x; P1[1] += uy * F1y; P1[2] += uz * F1z;
            P2[0] += ux * F2x; P2[1] += uy * F2y; P2[2] += uz * F2z;
            P1[3] += R(0.5) * (ux * F1y + uy * F1x); P2[3] += R(0.5) * (ux * F2y + uy * F2x);
            P1[4] += R(0.5) * (ux * F1z + uz * F1x); P2[4] += R(0.5) * (ux * F2z + uz * F2x);
            P1[5] += R(0.5) * (uy * F1z + uz * F1y); P2[5] += R(0.5) * (uy * F2z + uz * F2y);
        }
        P1[4] -= r1 * ux * uz; P2[4] -= r2 * ux * uz;
        P1[5] -= r1 * uy * uz; P2[5] -= r2 * uy * uz;
        t1 = (P1[0] + P1[1] + P1[2]) / R(3);
        t2 = (P2[0] + P2[1] + P2[2]) / R(3);
        if (REG == 2) { th1.finish(r1, ux, uy, uz); th2.finish(r2, ux, uy, uz); }
    }
    // rest population (k_0 = 12)
    {
        const R w0 = w<R>(0);
        R o1, o2v;
        if (!REG) {
            const float2 f0 = s0[0];
            o1 = rq1 * R(12) * (A1 - keep1 * Au) + keep1 * f0.x;
            o2v = rq2 * R(12) * (A2 - keep2 * Au) + keep2 * f0.y;
        } else {
            o1 = rq1 * R(12) * A1 - keep1 * R(1.5) * t1;
            o2v = rq2 * R(12) * A2 - keep2 * R(1.5) * t2;
        }
        if constexpr (FORCE == FORCE_GUO) {   // forcing term of the rest population: w_0 (-3 u*.F)
            o1 += cf1 * (R(-1) * uF1);
            o2v += cf2 * (R(-1) * uF2);
        }
        if constexpr (Store<S>::kRel) {
            const float2 iv = rinv[sl_c][ly][lx];   // 1/rho of the cell itself; 1/w_0 = 3
            Store<S>::store2(o, o1, o2v, R(3) * iv.x, R(3) * iv.y);
            state_ref(fout, p.ref_off)[cell] = rr;
        } else if constexpr (Store<S>::kDev) {
            Store<S>::store2_d(o, o1 - w0 * dc1, o2v - w0 * dc2);
        } else {
            Store<S>::store2(o, o1, o2v, w0 * ref0, w0 * ref0);
        }
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const R cu = cdot<R>(i, ux, uy, uz);
        const R c1 = cdot<R>(i, v1x, v1y, v1z);
        const R c2 = cdot<R>(i, v2x, v2y, v2z);
        // E = A + 4.5 (c.v)^2, O = (c.v) (B + 4.5 (c.v)^2): f^eq_+- = rho w (E +- O)
        const R E1 = A1 + R(4.5) * c1 * c1, O1 = c1 * (B1 + R(4.5) * c1 * c1);
        const R E2 = A2 + R(4.5) * c2 * c2, O2 = c2 * (B2 + R(4.5) * c2 * c2);
        const R rw1 = rq1 * R(k36(i)), rw2 = rq2 * R(k36(i));
        R o1p, o1m, o2p, o2m;
        if (!REG) {
            // f* = f^eq(v) + keep (f - f^eq(u)); f^eq(u) shares its polynomial between components
            const R Eu = Au + R(4.5) * cu * cu, Ou = cu * (Bu + R(4.5) * cu * cu);
            R P1e = rw1 * (E1 - keep1 * Eu), M1 = rw1 * (O1 - keep1 * Ou);
            R P2e = rw2 * (E2 - keep2 * Eu), M2 = rw2 * (O2 - keep2 * Ou);
            if constexpr (Store<S>::kDev) { P1e -= w<R>(i) * dc1; P2e -= w<R>(i) * dc2; }
            const float2 fp = s0[i * kThreadsF], fm = s0[(i + 1) * kThreadsF];
            o1p = P1e + M1 + keep1 * fp.x;
            o1m = P1e - M1 + keep1 * fm.x;
            o2p = P2e + M2 + keep2 * fp.y;
            o2m = P2e - M2 + keep2 * fm.y;
        } else {
            // f* = f^eq(v) + keep (k_i / 8) (c c : Pi - tr(Pi) / 3)
            R cc1 = 0, cc2 = 0;
            if (cx(i)) { cc1 += P1[0]; cc2 += P2[0]; }
            if (cy(i)) { cc1 += P1[1]; cc2 += P2[1]; }
            if (cz(i)) { cc1 += P1[2]; cc2 += P2[2]; }
            if (cx(i) && cy(i)) { const R sg = cx(i) == cy(i) ? R(2) : R(-2); cc1 += sg * P1[3]; cc2 += sg * P2[3]; }
            if (cx(i) && cz(i)) { const R sg = cx(i) == cz(i) ? R(2) : R(-2); cc1 += sg * P1[4]; cc2 += sg * P2[4]; }
            if (cy(i) && cz(i)) { const R sg = cy(i) == cz(i) ? R(2) : R(-2); cc1 += sg * P1[5]; cc2 += sg * P2[5]; }
            R n1 = keep1 * (R(k36(i)) * R(0.125)) * (cc1 - t1);
            R n2 = keep2 * (R(k36(i)) * R(0.125)) * (cc2 - t2);
            if constexpr (Store<S>::kDev) { n1 -= w<R>(i) * dc1; n2 -= w<R>(i) * dc2; }
            // third-order part, odd in c_i: + for i, - for opp(i)
            const R m1 = REG == 2 ? keep1 * th1.odd(i) : R(0);
            const R m2 = REG == 2 ? keep2 * th2.odd(i) : R(0);
            o1p = rw1 * (E1 + O1) + n1 + m1;
            o1m = rw1 * (E1 - O1) + n1 - m1;
            o2p = rw2 * (E2 + O2) + n2 + m2;
            o2m = rw2 * (E2 - O2) + n2 - m2;
        }
        if constexpr (FORCE == FORCE_GUO) {
            const R kq = R(k36(i)) / R(36);
            const R cF1 = cdot<R>(i, F1x, F1y, F1z), cF2 = cdot<R>(i, F2x, F2y, F2z);
            const R e1 = cf1 * kq * (R(9) * cu * cF1 - R(3) * uF1), d1 = cf1 * kq * (R(3) * cF1);
            const R e2 = cf2 * kq * (R(9) * cu * cF2 - R(3) * uF2), d2 = cf2 * kq * (R(3) * cF2);
            o1p += e1 + d1; o1m += e1 - d1;
            o2p += e2 + d2; o2m += e2 - d2;
        }
        const size_t ip = 2 * (size_t)((unsigned)i * N32), im = 2 * (size_t)((unsigned)(i + 1) * N32);
        if constexpr (Store<S>::kRel) {
            // destinations: x + c_i for i, x - c_i for opp(i), or x across a wall
            const bool wp = (cz(i) == -1 && lo_wall) || (cz(i) == 1 && hi_wall) || ((lw >> (i + 1)) & 1u);
            const bool wm = (cz(i) == 1 && lo_wall) || (cz(i) == -1 && hi_wall) || ((lw >> i) & 1u);
            const int slp = cz(i) == -1 ? sl_m : (cz(i) == 1 ? sl_p : sl_c);
            const int slm = cz(i) == -1 ? sl_p : (cz(i) == 1 ? sl_m : sl_c);
            const float2 dp = wp ? rinv[sl_c][ly][lx] : rinv[slp][ly + cy(i)][lx + cx(i)];
            const float2 dm = wm ? rinv[sl_c][ly][lx] : rinv[slm][ly - cy(i)][lx - cx(i)];
            const R sk = R(36 / k36(i));   // 1 / w_i: the code parameter is 1 / (w_i rho~)
            Store<S>::store2(o + ip, o1p, o2p, sk * dp.x, sk * dp.y);
            Store<S>::store2(o + im, o1m, o2m, sk * dm.x, sk * dm.y);
        } else if constexpr (Store<S>::kDev) {
            Store<S>::store2_d(o + ip, o1p, o2p);
            Store<S>::store2_d(o + im, o1m, o2m);
        } else {
            const R ref = w<R>(i) * ref0;
            Store<S>::store2(o + ip, o1p, o2p, ref, ref);
            Store<S>::store2(o + im, o1m, o2m, ref, ref);
        }
    }
}

// Interior part of plane zp for this thread's column: rho^1, rho^2 into ring
// slot `slot`; when st >= 0 the populations and momentum into stash slot st.
// A solid site of a mask (solid) presents its wall density wd instead.
template <int S>
__device__ __forceinline__ void interior_plane(const typename Store<S>::T *__restrict__ f,
                                               const Phys<typename Store<S>::R> &p, FusedSmem<typename Store<S>::R> &sm,
                                               InvRing *inv,
                                               int slot, int st, const PlaneRef &pr, const typename Store<S>::R (&v)[Q2],
                                               bool solid = false, float2 wd = make_float2(0.f, 0.f))
{
    using R = typename Store<S>::R;
    const int tid = threadIdx.x;
    const int lx = tid % kTX + 1, ly = tid / kTX + 1;
    R r1 = p.rho_s[0], r2 = p.rho_s[1];
    if (solid) {
        r1 = wd.x;
        r2 = wd.y;
    } else if (!pr.constant) {
        R a1, a2, jx, jy, jz;
        sums(v, a1, a2, jx, jy, jz);
        if constexpr (Store<S>::kDev) { a1 += p.rho0; a2 += p.rho0; }   // sum_i w_i rho0 = rho0
        if (pr.ghost) {
            r1 += a1; r2 += a2;
        } else {
            r1 = a1; r2 = a2;
            if (st >= 0) {
#pragma unroll
                for (int k = 0; k < Q; ++k) sm.stash[st][k][tid] = make_float2(v[k], v[Q + k]);
                sm.mom[st][0][tid] = jx; sm.mom[st][1][tid] = jy; sm.mom[st][2][tid] = jz;
            }
        }
    }
    put_ring<S>(sm, inv, slot, ly, lx, r1, r2);
}

// Halo densities of a plane in ring slot `slot` from the partials of the
// population groups (mask: the kernel runs a solid mask, whose solid halo
// cells are marked in hsolid).
template <int S, class R>
__device__ __forceinline__ void halo_combine(const Phys<R> &p, FusedSmem<R> &sm, InvRing *inv, int slot, int hs,
                                             const PlaneRef &pr, int h, int hx, int hy, bool mask = false)
{
    R r1, r2;
    if (pr.constant) {
        r1 = p.rho_s[0];
        r2 = p.rho_s[1];
    } else {
        r1 = sm.hpart[hs][0][0][h] + sm.hpart[hs][1][0][h] + sm.hpart[hs][2][0][h];
        r2 = sm.hpart[hs][0][1][h] + sm.hpart[hs][1][1][h] + sm.hpart[hs][2][1][h];
        // partials of deviations (a solid halo cell's first partial is its wall density)
        if constexpr (Store<S>::kDev) {
            if (!(mask && sm.hsolid[hs][h])) { r1 += p.rho0; r2 += p.rho0; }
        }
        if (pr.ghost) { r1 += p.rho_s[0]; r2 += p.rho_s[1]; }
    }
    put_ring<S>(sm, inv, slot, hy, hx, r1, r2);
}

// MASK: staircase walls given as a mask of solid sites (the lattice is then
// periodic along z).  links holds every cell's link word (bit 0: the cell is
// solid; bit i: x - c_i is solid, so that link bounces back) and wrho the
// densities (rho^1, rho^2) that each solid site presents to Eq. 13.  The link
// words of the planes a thread gathers are loaded one plane ahead; a solid
// site puts its wall density into the ring (a solid halo cell through its
// first partial, the others zero) and stores zero populations.
template <int S, int REG, bool WALLZ, bool MASK, int FORCE>
__global__ void __launch_bounds__(kThreadsF, 2)
k_step_fused(const typename Store<S>::T *__restrict__ fin, typename Store<S>::T *__restrict__ fout,
             Phys<typename Store<S>::R> p, int ntx, int lz, typename Store<S>::R *__restrict__ s_out,
             const unsigned *__restrict__ links, const float2 *__restrict__ wrho)
{
    using R = typename Store<S>::R;
    static_assert(sizeof(R) == sizeof(float), "the fused step runs FP32 arithmetic");
    static_assert(!(MASK && WALLZ), "a solid mask needs a lattice periodic along z");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<R> &sm = *reinterpret_cast<FusedSmem<R> *>(smem_raw);
    InvRing *inv = reinterpret_cast<InvRing *>(smem_raw + sizeof(FusedSmem<R>));   // *_REL formats only
    const int tid = threadIdx.x;
    const int tx0 = (blockIdx.x % ntx) * kTX;
    const int ty0 = (blockIdx.x / ntx) * kTY;
    const int z0 = blockIdx.y * lz;
    const int z1 = min(z0 + lz, p.nz);
    const int lx = tid % kTX, ly = tid / kTX;
    const int x = tx0 + lx, y = ty0 + ly;
    const bool active = x < p.nx && y < p.ny;
    // interior column (wrapped so that ragged tiles fill their ring slots
    // with the periodic images their active neighbours read)
    const Col ci = make_col((tx0 + lx) % p.nx, (ty0 + ly) % p.ny, p.nx, p.ny);
    auto halo_pos = [](int hh, int &hx, int &hy) {
        if (hh < kTX + 2) { hx = hh; hy = 0; }
        else if (hh < 2 * (kTX + 2)) { hx = hh - (kTX + 2); hy = kTY + 1; }
        else { const int k = hh - 2 * (kTX + 2); hx = k < kTY ? 0 : kTX + 1; hy = 1 + (k % kTY); }
    };
    auto halo_col = [&](int hx_, int hy_) {
        int gx = (tx0 - 1 + hx_) % p.nx; if (gx < 0) gx += p.nx;
        int gy = (ty0 - 1 + hy_) % p.ny; if (gy < 0) gy += p.ny;
        return make_col(gx, gy, p.nx, p.ny);
    };
    // halo cell h = tid (< 84) of this thread for the full gathers of the
    // prologue and for completing the halo densities
    const int h = tid % kHalo;
    int hx, hy;
    halo_pos(h, hx, hy);
    const Col ch = halo_col(hx, hy);
    // partial-gather task (cell ht, population group g): every warp takes 25-26
    // consecutive row-halo tasks (coalesced) and 6 of the 48 side-column tasks
    // (one scattered sector per load), so no warp carries the side columns alone
    constexpr int kRowCells = 2 * (kTX + 2), kSideCells = 2 * kTY;
    constexpr int kRowTasks = kGroups * kRowCells, kSideTasks = kGroups * kSideCells;
    constexpr int kWarps = kThreadsF / 32;
    static_assert(kSideTasks % kWarps == 0, "side tasks spread evenly over the warps");
    constexpr int kSidePerWarp = kSideTasks / kWarps, kRowBase = kRowTasks / kWarps, kRowExtra = kRowTasks % kWarps;
    static_assert(kRowBase + (kRowExtra ? 1 : 0) + kSidePerWarp <= 32, "halo tasks fit a warp");
    int ht = 0, g = 0;
    bool has_halo = false;
    {
        const int w = tid >> 5, lane = tid & 31;
        const int nrow = kRowBase + (w < kRowExtra ? 1 : 0);
        const int row0 = w * kRowBase + (w < kRowExtra ? w : kRowExtra);
        if (lane < nrow) {
            const int t = row0 + lane;
            g = t / kRowCells; ht = t % kRowCells; has_halo = true;
        } else if (lane - nrow < kSidePerWarp) {
            const int t = w * kSidePerWarp + (lane - nrow);
            g = t / kSideCells; ht = kRowCells + t % kSideCells; has_halo = true;
        }
    }
    int htx, hty;
    halo_pos(ht, htx, hty);
    const Col cht = halo_col(htx, hty);

    // ring slot of plane q: (q - z0 + 1) & 3; stash, moment and halo-partial
    // slot of plane q: (q - z0) & 1.
    // prologue: planes z0-1 and z0 in full, halo partials of z0+1
    // link word of column c at plane pr (0 without a mask)
    auto link_of = [&](const PlaneRef &pr, const Col &c) -> unsigned {
        return MASK ? __ldg(links + (unsigned)(pr.zc + c.yo[1] + c.xo[1])) : 0u;
    };
    // wall density of a solid site: rho_s (point-wise potential), or the
    // refreshed mean of the mirror model
    auto wall_rho = [&](const PlaneRef &pr, const Col &c) -> float2 {
        if (!p.wall_mirror) return make_float2((float)p.rho_s[0], (float)p.rho_s[1]);
        return __ldg(wrho + (unsigned)(pr.zc + c.yo[1] + c.xo[1]));
    };
    unsigned lwA = 0;   // link word of the thread's column at plane z (its collision)
    for (int q = z0 - 1; q <= z0; ++q) {
        const PlaneRef pr = plane_ref<WALLZ>(p, q);
        const unsigned lw = link_of(pr, ci);
        if (q == z0) lwA = lw;
        R v[Q2];
        if (!pr.constant) GatherAll<S, 0>::run(fin, p.N, gather_ref<S>(fin, p, pr, ci), pr, ci, lw, v);
        const bool sol = MASK && (lw & 1u);
        interior_plane<S>(fin, p, sm, inv, q - z0 + 1, q == z0 ? 0 : -1, pr, v, sol,
                          sol ? wall_rho(pr, ci) : make_float2(0.f, 0.f));
        if (tid < kHalo) {
            R r1 = p.rho_s[0], r2 = p.rho_s[1];
            const unsigned hl = link_of(pr, ch);
            if (MASK && (hl & 1u)) {
                const float2 wd = wall_rho(pr, ch);
                r1 = wd.x;
                r2 = wd.y;
            } else if (!pr.constant) {
                R hv[Q2];
                GatherAll<S, 0>::run(fin, p.N, gather_ref<S>(fin, p, pr, ch), pr, ch, hl, hv);
                R a1, a2, jx, jy, jz;
                sums(hv, a1, a2, jx, jy, jz);
                if constexpr (Store<S>::kDev) { a1 += p.rho0; a2 += p.rho0; }
                if (pr.ghost) { r1 += a1; r2 += a2; } else { r1 = a1; r2 = a2; }
            }
            put_ring<S>(sm, inv, q - z0 + 1, hy, hx, r1, r2);
        }
    }
    // halo partials of plane z0+1; a solid halo cell gives its wall density
    // as the first group's partial and zeros as the others
    auto halo_task = [&](const PlaneRef &pr, unsigned hl, int slot) {
        R hv[kPer];
        R s1 = 0, s2 = 0;
        if (MASK && (hl & 1u)) {
            if (g == 0) {
                const float2 wd = wall_rho(pr, cht);
                s1 = wd.x;
                s2 = wd.y;
            }
        } else if (!pr.constant) {
            halo_load<S>(fin, p, pr, cht, hl, g, hv);
            halo_sum<S>(hv, g, s1, s2);
        }
        if (MASK && g == 0) sm.hsolid[slot][ht] = (hl & 1u) ? 1 : 0;
        sm.hpart[slot][g][0][ht] = s1;
        sm.hpart[slot][g][1][ht] = s2;
    };
    if (has_halo) {
        const PlaneRef pr = plane_ref<WALLZ>(p, z0 + 1);
        halo_task(pr, link_of(pr, cht), 1);
    }
    // interior populations of plane z0+1, in registers until the first iteration
    // Interior populations of plane z+1, in registers from the gathers issued
    // before the previous collision until phase A: decoded (v), or, in the
    // 16-bit instances that run periodic lattices without a mask (the ones
    // measured to gain from it), as stored (rv, with the reference densities
    // rrv), which keeps 19 registers instead of 38 live across the collision.
    constexpr bool kRaw = sizeof(typename Store<S>::Raw) < sizeof(float2) && !WALLZ && !MASK;
    R v[Q2];
    typename Store<S>::Raw rv[Q];
    float2 rrv = make_float2(0.f, 0.f);
    unsigned lwB, lwC = 0, hlw = 0;   // link words: column at z+1, z+2; halo task cell at z+2
    float2 wdB = make_float2(0.f, 0.f);   // wall density of the column at z+1 (a solid site)
    auto gather_interior = [&](const PlaneRef &pr, unsigned lw) {
        if constexpr (kRaw) {
            rrv = gather_ref<S>(fin, p, pr, ci);
            GatherRaw<S, 0>::run(fin, p.N, pr, ci, lw, rv);
        } else {
            GatherAll<S, 0>::run(fin, p.N, gather_ref<S>(fin, p, pr, ci), pr, ci, lw, v);
        }
    };
    {
        const PlaneRef pr = plane_ref<WALLZ>(p, z0 + 1);
        lwB = link_of(pr, ci);
        if (!pr.constant) gather_interior(pr, lwB);
        if (MASK) {
            if (lwB & 1u) wdB = wall_rho(pr, ci);
            const PlaneRef pr2 = plane_ref<WALLZ>(p, z0 + 2);
            lwC = link_of(pr2, ci);
            if (has_halo) hlw = link_of(pr2, cht);
        }
    }
    __syncthreads();

    const long long cell_xy = (long long)y * p.nx + x;
    for (int z = z0; z < z1; ++z) {
        const int k = z - z0;
        const int s_m = k & 3, s_c = (k + 1) & 3, s_p = (k + 2) & 3;
        // ---- phase A: plane z+1 from the registers filled during the previous
        //      collision; halo partial gathers of plane z+2
        const PlaneRef pr1 = plane_ref<WALLZ>(p, z + 1);
        const bool need2 = z + 2 <= z1;           // rho(z+2) feeds the collision of z+1
        const PlaneRef pr2 = plane_ref<WALLZ>(p, z + 2);
        R hv[kPer];
        const bool hsol = MASK && (hlw & 1u);   // the halo task's cell is a solid site
        float2 hwd = make_float2(0.f, 0.f);
        if (hsol && g == 0 && need2 && has_halo) hwd = wall_rho(pr2, cht);   // in flight with the gathers
        if (need2 && has_halo && !hsol && !pr2.constant) halo_load<S>(fin, p, pr2, cht, hlw, g, hv);
        if (tid < kHalo) halo_combine<S>(p, sm, inv, s_p, (k + 1) & 1, pr1, h, hx, hy, MASK);
        const bool sol = MASK && (lwB & 1u);
        if constexpr (kRaw) {
            if (!pr1.constant) decode_all<S>(rv, rrv, v);
        }
        interior_plane<S>(fin, p, sm, inv, s_p, z + 1 < z1 ? ((k + 1) & 1) : -1, pr1, v, sol, wdB);
        if (need2 && has_halo) {
            R s1 = 0, s2 = 0;
            if (hsol) {
                if (g == 0) {
                    s1 = hwd.x;
                    s2 = hwd.y;
                }
            } else if (!pr2.constant) {
                halo_sum<S>(hv, g, s1, s2);
            }
            if (MASK && g == 0) sm.hsolid[k & 1][ht] = hsol ? 1 : 0;
            sm.hpart[k & 1][g][0][ht] = s1;
            sm.hpart[k & 1][g][1][ht] = s2;
        }
        __syncthreads();
        // ---- phase B: the interior gathers of plane z+2 are issued first and
        //      stay in flight (in registers) during the collision of plane z
        if (z + 1 < z1 && !pr2.constant) gather_interior(pr2, lwC);
        unsigned lwD = 0;
        float2 wdC = make_float2(0.f, 0.f);
        if (MASK) {   // link words of plane z+3 (periodic z: always a lattice plane)
            const PlaneRef pr3 = plane_ref<WALLZ>(p, z + 3);
            lwD = link_of(pr3, ci);
            if (has_halo) hlw = link_of(pr3, cht);
            if (lwC & 1u) wdC = wall_rho(pr2, ci);   // the column at z+2 is a solid site
        }
        if (active)
            collide_cell<S, REG, FORCE>(fout, p, sm, inv, s_m, s_c, s_p, k & 1, (long long)z * p.nx * p.ny + cell_xy, s_out,
                                 WALLZ && z == 0, WALLZ && z == p.nz - 1, lwA);
        lwA = lwB;
        lwB = lwC;
        lwC = lwD;
        wdB = wdC;
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
    p.ref_off = h.ref_off;
    return p;
}

constexpr int kMaxAttrDevices = 64;

// Launch of one kernel instance.  The dynamic shared-memory size attribute
// belongs to the device context: each instance sets it once per device
// (several host threads may race to set the same value, which is harmless).
template <int S, int REG, bool WALLZ, bool MASK, int FORCE>
cudaError_t launch_inst(dim3 grid, cudaStream_t s, const typename Store<S>::T *fi, typename Store<S>::T *fo,
                        const Phys<typename Store<S>::R> &p, int ntx, int lz, typename Store<S>::R *s_out,
                        const unsigned *links, const float2 *wrho)
{
    static std::atomic<int> attr_set[kMaxAttrDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kMaxAttrDevices;
    if (!cached || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute((const void *)k_step_fused<S, REG, WALLZ, MASK, FORCE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<S>());
        if (e != cudaSuccess) return e;
        if (cached) attr_set[dev].store(1, std::memory_order_release);
    }
    k_step_fused<S, REG, WALLZ, MASK, FORCE><<<grid, kThreadsF, smem_bytes<S>(), s>>>(fi, fo, p, ntx, lz, s_out, links, wrho);
    return cudaSuccess;
}

template <int S, int REG, int FORCE>
cudaError_t launch_geom(const HostPhys &h, int lz, dim3 grid, cudaStream_t s, const typename Store<S>::T *fi,
                        typename Store<S>::T *fo, const Phys<typename Store<S>::R> &p, int ntx,
                        typename Store<S>::R *s_out)
{
    if (h.wall_z) return launch_inst<S, REG, true, false, FORCE>(grid, s, fi, fo, p, ntx, lz, s_out, nullptr, nullptr);
    if (h.links)
        return launch_inst<S, REG, false, true, FORCE>(grid, s, fi, fo, p, ntx, lz, s_out, h.links,
                                                       (const float2 *)h.wall_rho);
    return launch_inst<S, REG, false, false, FORCE>(grid, s, fi, fo, p, ntx, lz, s_out, nullptr, nullptr);
}

template <int S, int FORCE>
cudaError_t launch_coll(const HostPhys &h, int lz, dim3 grid, cudaStream_t s, const typename Store<S>::T *fi,
                        typename Store<S>::T *fo, const Phys<typename Store<S>::R> &p, int ntx,
                        typename Store<S>::R *s_out)
{
    switch (h.collision) {
    case LBM_REGULARIZED: return launch_geom<S, 1, FORCE>(h, lz, grid, s, fi, fo, p, ntx, s_out);
    case LBM_REGULARIZED3: return launch_geom<S, 2, FORCE>(h, lz, grid, s, fi, fo, p, ntx, s_out);
    default: return launch_geom<S, 0, FORCE>(h, lz, grid, s, fi, fo, p, ntx, s_out);
    }
}

// Wall densities of the mirror model under a mask (Eq. 13, modified model),
// refreshed before each fused step: first the densities of the fluid cells
// that have a solid neighbour, summed like the fused kernel sums its ring
// (same gathers, same grouping), into their own entries of wall_rho; then each
// solid site with a fluid neighbour takes the w_i-weighted mean of its fluid
// neighbours' densities plus rho_s.
// Three lanes per fluid cell (ten cells per warp), one population group each
// as in the halo partial gathers, so that the groups' loads are in flight
// together; the first lane combines the three partials in the halo order.
template <int S>
__global__ void __launch_bounds__(256)
k_wall_fluid_rho(const typename Store<S>::T *__restrict__ f, Phys<typename Store<S>::R> p,
                 const unsigned *__restrict__ links, const unsigned *__restrict__ cells, long long n,
                 float2 *__restrict__ wr)
{
    using R = typename Store<S>::R;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int g = lane % 3;
    const long long t = warp * 10 + lane / 3;
    const bool ok = lane < 30 && t < n;
    R s1 = 0, s2 = 0;
    unsigned c = 0;
    if (ok) {
        c = cells[t];
        const unsigned plane = (unsigned)p.nx * (unsigned)p.ny;
        const int z = (int)(c / plane);
        const unsigned rem = c - (unsigned)z * plane;
        const int y = (int)(rem / (unsigned)p.nx), x = (int)(rem - (unsigned)y * (unsigned)p.nx);
        const Col col = make_col(x, y, p.nx, p.ny);
        const PlaneRef pr = plane_ref<false>(p, z);
        R v[kPer];
        halo_load<S>(f, p, pr, col, __ldg(links + c), g, v);
        halo_sum<S>(v, g, s1, s2);
    }
    const unsigned full = 0xffffffffu;
    const R a1 = __shfl_down_sync(full, s1, 1), a2 = __shfl_down_sync(full, s2, 1);
    const R b1 = __shfl_down_sync(full, s1, 2), b2 = __shfl_down_sync(full, s2, 2);
    R d1 = s1 + a1 + b1, d2 = s2 + a2 + b2;
    if constexpr (Store<S>::kDev) { d1 += p.rho0; d2 += p.rho0; }   // the partials sum deviations
    if (ok && g == 0) wr[c] = make_float2(d1, d2);
}

template <int S>   // (instantiated per storage format's translation unit)
__global__ void __launch_bounds__(256)
k_wall_solid_rho(const unsigned char *__restrict__ solid, Phys<float> p, const unsigned *__restrict__ cells,
                 long long n, float2 *__restrict__ wr)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned c = cells[t];
    const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, nz = (unsigned)p.nz, plane = nx * ny;
    const unsigned z = c / plane, rem = c - z * plane, y = rem / nx, x = rem - y * nx;
    float num1 = 0, num2 = 0;
    int den36 = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const unsigned xn = (x + nx + cx(i)) % nx, yn = (y + ny + cy(i)) % ny, zn = (z + nz + cz(i)) % nz;
        const unsigned nb = (zn * ny + yn) * nx + xn;
        if (__ldg(solid + nb)) continue;
        const float k = (float)k36(i);
        const float2 r = wr[nb];
        num1 += k * r.x;
        num2 += k * r.y;
        den36 += k36(i);
    }
    wr[c] = make_float2((den36 ? num1 / (float)den36 : 0.f) + p.rho_s[0], (den36 ? num2 / (float)den36 : 0.f) + p.rho_s[1]);
}

template <int S>
cudaError_t fused_t(const HostPhys &h, const void *fin, void *fout, cudaStream_t s, cudaEvent_t *ev, void *s_out)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const Phys<R> p = make_phys_f<R>(h);
    const int ntx = (h.nx + kTX - 1) / kTX;
    const int nty = (h.ny + kTY - 1) / kTY;
    const int lz = fused_planes((long long)ntx * nty, h.nz, current_device_sms());
    const dim3 grid((unsigned)(ntx * nty), (unsigned)((h.nz + lz - 1) / lz));
    if (ev) cudaEventRecord(ev[0], s);
    const T *fi = (const T *)fin;
    T *fo = (T *)fout;
    if (h.links && h.wall_mirror && h.n_bsolid > 0) {
        float2 *wr = (float2 *)h.wall_rho;
        if (h.n_bfluid > 0)
            k_wall_fluid_rho<S><<<(unsigned)((h.n_bfluid + 79) / 80), 256, 0, s>>>(fi, p, h.links, h.bfluid,
                                                                                 h.n_bfluid, wr);
        k_wall_solid_rho<S><<<(unsigned)((h.n_bsolid + 255) / 256), 256, 0, s>>>(h.solid, make_phys_f<float>(h), h.bsolid,
                                                                             h.n_bsolid, wr);
    }
    const cudaError_t e = h.forcing == FORCE_GUO
                              ? launch_coll<S, FORCE_GUO>(h, lz, grid, s, fi, fo, p, ntx, (R *)s_out)
                              : launch_coll<S, FORCE_EDM>(h, lz, grid, s, fi, fo, p, ntx, (R *)s_out);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    return cudaGetLastError();
}

}  // namespace fused
}  // namespace lbm
