// D3Q19 lattice, storage formats and the per-cell physics shared by the
// library's kernels (Otomo et al., arXiv:1601.01237, Sec. 2).
//
// Direction order of this library: 0 = rest, then opposite pairs side by side
// (1,2) = +-x, (3,4) = +-y, (5,6) = +-z, then the twelve face diagonals as
// (7,8) (9,10) (11,12) (13,14) (15,16) (17,18).  opp(i) = i + 1 for odd i,
// i - 1 for even i > 0.  Weights: 1/3 rest, 1/18 axis links, 1/36 diagonals
// (the textbook D3Q19 set; the paper names the set but does not print it).
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

namespace lbm {

constexpr int Q = 19;

// Components of c_i, two bits per direction (value + 1), direction 0 in the
// lowest bits.
//            i:  0  1  2  3  4  5  6  7  8  9 10 11 12 13 14 15 16 17 18
//   cx        :  0  1 -1  0  0  0  0  1 -1  1 -1  1 -1  1 -1  0  0  0  0
//   cy        :  0  0  0  1 -1  0  0  1 -1 -1  1  0  0  0  0  1 -1  1 -1
//   cz        :  0  0  0  0  0  1 -1  0  0  0  0  1 -1 -1  1  1 -1 -1  1
__host__ __device__ constexpr uint64_t pack_dirs(const int (&v)[Q])
{
    uint64_t r = 0;
    for (int i = Q - 1; i >= 0; --i) r = (r << 2) | (uint64_t)(v[i] + 1);
    return r;
}
constexpr int kCX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kCY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kCZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
constexpr uint64_t kPackX = pack_dirs(kCX);
constexpr uint64_t kPackY = pack_dirs(kCY);
constexpr uint64_t kPackZ = pack_dirs(kCZ);

__host__ __device__ constexpr int cx(int i) { return (int)((kPackX >> (2 * i)) & 3u) - 1; }
__host__ __device__ constexpr int cy(int i) { return (int)((kPackY >> (2 * i)) & 3u) - 1; }
__host__ __device__ constexpr int cz(int i) { return (int)((kPackZ >> (2 * i)) & 3u) - 1; }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wd(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

template <class R>
__host__ __device__ constexpr R w(int i) { return (R)wd(i); }
// Weights as exact integer numerators over 36 (12, 2, 1): the collision forms
// rho w_i as (rho / 36) k_i, so that the FP32 weights sum to one exactly.  The
// rounded FP32 values of 1/3, 1/18, 1/36 sum to 1 + 1.5e-8, which would add
// that fraction of mass times 1/tau at every BGK collision.
__host__ __device__ constexpr int k36(int i) { return i == 0 ? 12 : (i < 7 ? 2 : 1); }
__host__ __device__ constexpr int ca(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }

// Third-order Hermite polynomials on D3Q19.  Of the ten H_abc, four vanish on
// the lattice (H_xxx, H_yyy, H_zzz because c^3 = c and 3 T0 = 1; H_xyz because
// no direction has three non-zero components).  The other six pair up along
// the axis a of the odd index, with b < c the two other axes:
//   H_abb + H_acc = c_a (c_b^2 + c_c^2 - 2 T0)   (the energy flux along a)
//   H_abb - H_acc = c_a (c_b^2 - c_c^2)
// which are w-orthogonal on the lattice with norms 2/27 and 6/27.  h3s3 is
// 3 (H_abb + H_acc) and h3d is H_abb - H_acc, both integers.
__host__ __device__ constexpr int h3s3(int i, int a)
{
    return ca(i, a) * (3 * (ca(i, (a + 1) % 3) * ca(i, (a + 1) % 3) + ca(i, (a + 2) % 3) * ca(i, (a + 2) % 3)) - 2);
}
__host__ __device__ constexpr int h3d(int i, int a)
{
    // b < c: (y, z) for a = x, (x, z) for a = y, (x, y) for a = z
    return ca(i, a) * (a == 0 ? cy(i) * cy(i) - cz(i) * cz(i)
                              : (a == 1 ? cx(i) * cx(i) - cz(i) * cz(i) : cx(i) * cx(i) - cy(i) * cy(i)));
}

// Third-order part of the regularized filter for one component: accumulate
// the sums of h3s3 f_i and h3d f_i over the directions (add3), then subtract
// the same moments of f^eq(rho, u) (the third-order equilibrium of Eq. 3 on
// D3Q19 has sum_i (H_abb + H_acc) f^eq_i = rho u_a (u_b^2 + u_c^2) / 2 and
// sum_i (H_abb - H_acc) f^eq_i = 3 rho u_a (u_b^2 - u_c^2) / 2) to get
//   S_a = sum_i (H_abb + H_acc)(f_i - f^eq_i),  D_a = sum_i (H_abb - H_acc)(f_i - f^eq_i).
// The projection of (f - f^eq)/w onto the six polynomials then gives
//   f^neq3_i = (k_i / 8) sum_a (S_a h3s3(i, a) + D_a h3d(i, a))
// (w_i = k_i / 36; coefficients 1/(2/27) and 1/(6/27) on the pair basis).
template <class R>
struct Third {
    R s[3], d[3];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) { s[a] = R(0); d[a] = R(0); }
    }
    __device__ __forceinline__ void add(int i, R f)
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (h3s3(i, a)) s[a] += R(h3s3(i, a)) * f;
            if (h3d(i, a)) d[a] += R(h3d(i, a)) * f;
        }
    }
    __device__ __forceinline__ void finish(R rho, R ux, R uy, R uz)
    {
        const R u[3] = {ux, uy, uz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R ub = u[a == 0 ? 1 : 0], uc = u[a == 2 ? 1 : 2];
            const R ra = rho * u[a];
            s[a] = s[a] * (R(1) / R(3)) - R(0.5) * ra * (ub * ub + uc * uc);
            d[a] = d[a] - R(1.5) * ra * (ub * ub - uc * uc);
        }
    }
    // f^neq3 of direction i (the opposite direction takes the negative)
    __device__ __forceinline__ R odd(int i) const
    {
        R r = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (h3s3(i, a)) r += R(h3s3(i, a)) * s[a];
            if (h3d(i, a)) r += R(h3d(i, a)) * d[a];
        }
        return R(k36(i)) * R(0.125) * r;
    }
};

// ---------------------------------------------------------------------------
// Load of one FP32 population pair (the input copy, never written during a
// launch) with two cache hints: a 256-byte L2 prefetch size (a warp's row of
// 32 pulled pairs is 256 bytes and spans one or two 256-byte blocks that the
// neighbouring rows and tiles pull from too) and evict-last priority in L1.
// Chosen by measurement at 512^3 (ms per step): 8.33 with a plain load, 8.25
// with the read-only path and the L2 hint, 8.14 with a coherent load and the
// L2 hint, 8.08 with both hints; L1 no-allocate or evict-first: 11.5-12.2.
// The L1 hit rate stays near 1 % with every variant, so the L1 hint's gain
// does not come from reuse in L1.
__device__ __forceinline__ float2 ld_pair_f32(const float *p)
{
    float2 v;
    asm("ld.global.L1::evict_last.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
// The same load for a pair of 16-bit values (32 bits).  At 256^3 (ms per
// step, FP16 / BF16 deviations): BGK 0.902 / 0.917 -> 0.888 / 0.897,
// regularized 1.084 / 1.078 -> 1.071 / 1.070; the 128-byte prefetch size or
// the read-only path with the 256-byte size gained less.
__device__ __forceinline__ unsigned ld_pair_b16(const void *p)
{
    unsigned v;
    asm("ld.global.L1::evict_last.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// ---------------------------------------------------------------------------
// Storage formats.  R = arithmetic type, T = stored type.
//
// Population layout: direction-major, x fastest, with the two components of a
// cell side by side: f^a_i(cell) is element 2 (i N + cell) + a.  A pull gather
// fetches both components of a direction with one vector load (8 bytes in
// FP32) and a collision stores them with one vector store.
//
// Every format codes a population with one parameter per component, derived
// from a reference density rho_ref:
//   load:  f = dec(s, d) with d = w_i rho_ref (Store::load, load2),
//   store: s = enc(f, e) with e = Store::enc(w_i rho_ref) (Store::store, store2).
// FP64 / FP32 store f itself and ignore the parameters.  The *_DEV formats
// keep d_i = f_i - w_i rho0 in 16 bits (rho_ref = rho0 of the lattice).  The
// *_REL formats keep the relative deviation s_i = f_i / (w_i rho~) - 1 in 16
// bits, where rho~ is the density, at the step that produced it, of the cell
// that reads the population next (its destination): the writer knows it from
// the interaction stencil, and every cell stores its own rho~ (FP32, both
// components) beside the populations, so the reader decodes the 19
// populations it gathers with its own one reference.  A population at rest in
// a stationary bulk codes to 0 exactly, and both phases of a droplet keep the
// full 16-bit precision of s.
enum StorageKind { ST_F64 = 0, ST_F32 = 1, ST_F16_DEV = 2, ST_BF16_DEV = 3, ST_F16_REL = 4, ST_BF16_REL = 5 };

__host__ __device__ __forceinline__ long long pair_index(int i, long long cell, long long N)
{
    return 2 * ((long long)i * N + cell);
}

template <int S> struct Store;

template <> struct Store<ST_F64> {
    using T = double;
    using R = double;
    static constexpr bool kRel = false;
    static constexpr bool kDev = false;
    __device__ static __forceinline__ R enc(R wr) { return wr; }
    __device__ static __forceinline__ R load(const T *p, R) { return __ldg(p); }
    __device__ static __forceinline__ void store(T *p, R v, R) { *p = v; }
    __device__ static __forceinline__ void load2(const T *p, R, R, R &a, R &b)
    {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        a = v.x; b = v.y;
    }
    __device__ static __forceinline__ void store2(T *p, R a, R b, R, R) { *reinterpret_cast<double2 *>(p) = make_double2(a, b); }
};
template <> struct Store<ST_F32> {
    using T = float;
    using R = float;
    static constexpr bool kRel = false;
    static constexpr bool kDev = false;
    __device__ static __forceinline__ R enc(R wr) { return wr; }
    __device__ static __forceinline__ R load(const T *p, R) { return __ldg(p); }
    __device__ static __forceinline__ void store(T *p, R v, R) { *p = v; }
    __device__ static __forceinline__ void load2(const T *p, R, R, R &a, R &b)
    {
        const float2 v = ld_pair_f32(p);
        a = v.x; b = v.y;
    }
    __device__ static __forceinline__ void store2(T *p, R a, R b, R, R) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
    // a loaded pair as it is stored (Raw), decoded later (decode2): load2 in two halves
    using Raw = float2;
    __device__ static __forceinline__ Raw load_raw(const T *p) { return ld_pair_f32(p); }
    __device__ static __forceinline__ void decode2(Raw r, R, R, R &a, R &b) { a = r.x; b = r.y; }
};

// 16-bit conversions of the two formats.
struct H16 {
    using T = __half;
    using T2 = __half2;
    __device__ static __forceinline__ float to_f(T v) { return __half2float(v); }
    __device__ static __forceinline__ T from_f(float v) { return __float2half_rn(v); }
    __device__ static __forceinline__ void unpack(unsigned u, float &a, float &b)
    {
        __half2 v;
        memcpy(&v, &u, sizeof v);
        a = __low2float(v); b = __high2float(v);
    }
    __device__ static __forceinline__ T2 pack(float a, float b) { return __halves2half2(from_f(a), from_f(b)); }
};
struct B16 {
    using T = __nv_bfloat16;
    using T2 = __nv_bfloat162;
    __device__ static __forceinline__ float to_f(T v) { return __bfloat162float(v); }
    __device__ static __forceinline__ T from_f(float v) { return __float2bfloat16_rn(v); }
    __device__ static __forceinline__ void unpack(unsigned u, float &a, float &b)
    {
        __nv_bfloat162 v;
        memcpy(&v, &u, sizeof v);
        a = __low2float(v); b = __high2float(v);
    }
    __device__ static __forceinline__ T2 pack(float a, float b) { return __halves2bfloat162(from_f(a), from_f(b)); }
};

// Deviation d = f - w rho0 (parameters: w rho0 for both directions).
template <class C> struct StoreDev {
    using T = typename C::T;
    using R = float;
    static constexpr bool kRel = false;
    static constexpr bool kDev = true;
    __device__ static __forceinline__ R enc(R wr) { return wr; }
    __device__ static __forceinline__ R load(const T *p, R d) { return C::to_f(__ldg(p)) + d; }
    __device__ static __forceinline__ void store(T *p, R v, R e) { *p = C::from_f(v - e); }
    __device__ static __forceinline__ void load2(const T *p, R da, R db, R &a, R &b)
    {
        C::unpack(ld_pair_b16(p), a, b);
        a += da; b += db;
    }
    __device__ static __forceinline__ void store2(T *p, R a, R b, R ea, R eb)
    {
        *reinterpret_cast<typename C::T2 *>(p) = C::pack(a - ea, b - eb);
    }
    using Raw = unsigned;
    __device__ static __forceinline__ Raw load_raw(const T *p) { return ld_pair_b16(p); }
    __device__ static __forceinline__ void decode2(Raw r, R da, R db, R &a, R &b)
    {
        C::unpack(r, a, b);
        a += da; b += db;
    }
    // the deviations d themselves (the fused step computes in d = f - w rho0)
    __device__ static __forceinline__ void load2_d(const T *p, R &a, R &b) { C::unpack(ld_pair_b16(p), a, b); }
    __device__ static __forceinline__ void decode2_d(Raw r, R &a, R &b) { C::unpack(r, a, b); }
    __device__ static __forceinline__ void store2_d(T *p, R a, R b)
    {
        *reinterpret_cast<typename C::T2 *>(p) = C::pack(a, b);
    }
};
// Relative deviation s = f / (w rho~) - 1 (load parameter d = w rho~, store
// parameter e = 1 / (w rho~)).
template <class C> struct StoreRel {
    using T = typename C::T;
    using R = float;
    static constexpr bool kRel = true;
    static constexpr bool kDev = false;
    __device__ static __forceinline__ R enc(R wr) { return __frcp_rn(wr); }
    __device__ static __forceinline__ R load(const T *p, R d) { return fmaf(d, C::to_f(__ldg(p)), d); }
    __device__ static __forceinline__ void store(T *p, R v, R e) { *p = C::from_f(fmaf(v, e, -1.0f)); }
    __device__ static __forceinline__ void load2(const T *p, R da, R db, R &a, R &b)
    {
        float sa, sb;
        C::unpack(ld_pair_b16(p), sa, sb);
        a = fmaf(da, sa, da); b = fmaf(db, sb, db);
    }
    __device__ static __forceinline__ void store2(T *p, R a, R b, R ea, R eb)
    {
        *reinterpret_cast<typename C::T2 *>(p) = C::pack(fmaf(a, ea, -1.0f), fmaf(b, eb, -1.0f));
    }
    using Raw = unsigned;
    __device__ static __forceinline__ Raw load_raw(const T *p) { return ld_pair_b16(p); }
    __device__ static __forceinline__ void decode2(Raw r, R da, R db, R &a, R &b)
    {
        float sa, sb;
        C::unpack(r, sa, sb);
        a = fmaf(da, sa, da); b = fmaf(db, sb, db);
    }
};
template <> struct Store<ST_F16_DEV> : StoreDev<H16> {};
template <> struct Store<ST_BF16_DEV> : StoreDev<B16> {};
template <> struct Store<ST_F16_REL> : StoreRel<H16> {};
template <> struct Store<ST_BF16_REL> : StoreRel<B16> {};

// ---------------------------------------------------------------------------
// Kernel-side parameters (by value).
template <class R>
struct Phys {
    int nx, ny, nz;
    long long N;            // nx*ny*nz
    int wall_z;             // 1: half-way bounce-back walls at z = -1/2 and nz - 1/2
    int wall_mirror;        // 1: rho' = mirror + rho_s, 0: rho' = rho_s
    R omega[2];             // 1 / tau_a
    R G12, G21;             // G^{12}, G^{21} of Eq. 7 (signed)
    R gext[3];
    R rho_s[2];
    R rho0;                 // reference density of deviation storage (0 otherwise)
    const unsigned char *solid = nullptr;   // N flags, 1 = solid site (nullptr without a mask)
    long long ref_off = 0;  // *_REL formats: byte offset of the per-cell reference
                            // densities (float2 per cell) from the state's base
};

// Reference densities of a *_REL state (N pairs (rho~1, rho~2) behind the
// populations, at byte offset ref_off).
template <class T>
__device__ __forceinline__ const float2 *state_ref(const T *state, long long ref_off)
{
    return reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(state) + ref_off);
}
template <class T>
__device__ __forceinline__ float2 *state_ref(T *state, long long ref_off)
{
    return reinterpret_cast<float2 *>(reinterpret_cast<char *>(state) + ref_off);
}

// Third-order equilibrium of Eq. 3 with T0 = 1/3, for direction i and its
// opposite at once: f^eq_i = rho w_i (E + O), f^eq_opp(i) = rho w_i (E - O) with
//   E = 1 - u^2/(2T0) + (c.u)^2/(2T0^2)
//   O = (c.u)/T0 - (c.u) u^2/(2T0^2) + (c.u)^3/(6T0^3).
template <class R>
__device__ __forceinline__ void feq_pair(R rw, R cu, R usq, R &fp, R &fm)
{
    const R cu2 = cu * cu;
    const R E = R(1) - R(1.5) * usq + R(4.5) * cu2;
    const R O = cu * (R(3) - R(4.5) * usq + R(4.5) * cu2);
    fp = rw * (E + O);
    fm = rw * (E - O);
}

template <class R>
__device__ __forceinline__ R cdot(int i, R ux, R uy, R uz)
{
    R r = R(0);
    if (cx(i) == 1) r += ux; else if (cx(i) == -1) r -= ux;
    if (cy(i) == 1) r += uy; else if (cy(i) == -1) r -= uy;
    if (cz(i) == 1) r += uz; else if (cz(i) == -1) r -= uz;
    return r;
}

// Forcing schemes of the Sec. 2 forcing term (the paper cites the scheme
// without printing it; two readings are built):
//   FORCE_EDM: exact difference of equilibria, F_i = f^eq_i(rho, u + g) - f^eq_i(rho, u),
//              f^eq at the mixture velocity u of Eq. 6;
//   FORCE_GUO: Guo, Zheng & Shi (2002), per component with the common
//              equilibrium velocity u* = u + g/2 of Eqs. 8-9 and
//              F_i = w_i [(c_i - u*)/T0 + (c_i.u*) c_i / T0^2] . rho g.
enum ForcingKind { FORCE_EDM = 0, FORCE_GUO = 1 };

// Collision of one component in place: f[] holds the pre-collision f_i^a and
// receives the post-collision f*_i^a (Eq. 1 with Eq. 2, or Eq. 10).
// Exact-difference forcing (FORCE = FORCE_EDM; u = mixture velocity, g = g^a):
//   BGK (REG = 0):         f* = f^eq(u + g) + (1 - 1/tau) (f - f^eq(u))
//   regularized (REG = 1): f* = f^eq(u + g) + (1 - 1/tau) w_i/(2 T0^2) Q_i : Pi^neq,
//                 Pi^neq = sum_i c_i c_i f_i - rho (T0 I + u u);
//                 w_i/(2 T0^2) = k_i / 8 and Q_i : Pi = c_i c_i : Pi - tr(Pi)/3.
//   REG = 2: the regularized f^neq plus its third-order part (struct Third).
// Guo forcing (FORCE = FORCE_GUO; u = u* = u + g/2 of the mixture, g = g^a):
//   BGK:         f* = f^eq(u*) + (1 - 1/tau) (f - f^eq(u*)) + (1 - 1/(2 tau)) F
//   regularized: f* = f^eq(u*) + (1 - 1/tau) P[f - f^eq(u*) + F/2] + F/2, P the
//                projection above (Pi^neq gains (u* F + F u*)/2, the second
//                moment of F/2; F has no third-order part).
template <class R, int REG, int FORCE = FORCE_EDM>
__device__ __forceinline__ void collide(R (&f)[Q], R rho, R ux, R uy, R uz,
                                        R gx, R gy, R gz, R omega)
{
    if (FORCE == FORCE_GUO) {
        const R usq = ux * ux + uy * uy + uz * uz;
        const R keep = R(1) - omega;
        const R rq = rho / R(36);
        const R Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
        const R uF = ux * Fx + uy * Fy + uz * Fz;
        const R cf = REG ? R(0.5) : R(1) - R(0.5) * omega;   // weight of the forcing term
        // F_i = (k_i / 36) (even_i +- odd_i): even = 9 (c.u)(c.F) - 3 u.F, odd = 3 c.F
        R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0, t = 0;
        Third<R> th;
        if (REG) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const R v = f[i];
                if (cx(i)) pxx += v;
                if (cy(i)) pyy += v;
                if (cz(i)) pzz += v;
                if (cx(i) && cy(i)) { if (cx(i) == cy(i)) pxy += v; else pxy -= v; }
                if (cx(i) && cz(i)) { if (cx(i) == cz(i)) pxz += v; else pxz -= v; }
                if (cy(i) && cz(i)) { if (cy(i) == cz(i)) pyz += v; else pyz -= v; }
            }
            const R T0 = R(1) / R(3);
            // Pi of f - f^eq(u*) + F/2
            pxx += -rho * (T0 + ux * ux) + ux * Fx;
            pyy += -rho * (T0 + uy * uy) + uy * Fy;
            pzz += -rho * (T0 + uz * uz) + uz * Fz;
            pxy += -rho * ux * uy + R(0.5) * (ux * Fy + uy * Fx);
            pxz += -rho * ux * uz + R(0.5) * (ux * Fz + uz * Fx);
            pyz += -rho * uy * uz + R(0.5) * (uy * Fz + uz * Fy);
            t = (pxx + pyy + pzz) / R(3);
            if (REG == 2) {
                th.zero();
#pragma unroll
                for (int i = 1; i < Q; ++i) th.add(i, f[i]);
                th.finish(rho, ux, uy, uz);
            }
        }
        {
            const R e0 = rq * R(12) * (R(1) - R(1.5) * usq);
            const R F0 = R(12) / R(36) * (R(-3) * uF);
            f[0] = REG ? e0 + keep * (R(-1.5) * t) + cf * F0 : e0 + keep * (f[0] - e0) + cf * F0;
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const R cu = cdot<R>(i, ux, uy, uz);
            const R cF = cdot<R>(i, Fx, Fy, Fz);
            R ep, em;
            feq_pair<R>(rq * R(k36(i)), cu, usq, ep, em);
            const R kq = R(k36(i)) / R(36);
            const R Fe = kq * (R(9) * cu * cF - R(3) * uF), Fo = kq * (R(3) * cF);
            if (!REG) {
                f[i] = ep + keep * (f[i] - ep) + cf * (Fe + Fo);
                f[i + 1] = em + keep * (f[i + 1] - em) + cf * (Fe - Fo);
            } else {
                R cc = R(0);
                if (cx(i)) cc += pxx;
                if (cy(i)) cc += pyy;
                if (cz(i)) cc += pzz;
                if (cx(i) && cy(i)) cc += (cx(i) == cy(i) ? R(2) : R(-2)) * pxy;
                if (cx(i) && cz(i)) cc += (cx(i) == cz(i) ? R(2) : R(-2)) * pxz;
                if (cy(i) && cz(i)) cc += (cy(i) == cz(i) ? R(2) : R(-2)) * pyz;
                const R fneq = R(k36(i)) * R(0.125) * (cc - t);
                const R f3 = REG == 2 ? th.odd(i) : R(0);
                f[i] = ep + keep * (fneq + f3) + cf * (Fe + Fo);
                f[i + 1] = em + keep * (fneq - f3) + cf * (Fe - Fo);
            }
        }
        return;
    }
    const R usq = ux * ux + uy * uy + uz * uz;
    const R vx = ux + gx, vy = uy + gy, vz = uz + gz;
    const R vsq = vx * vx + vy * vy + vz * vz;
    const R keep = R(1) - omega;
    const R rq = rho / R(36);
    if (!REG) {
        {
            const R e0 = rq * R(12) * (R(1) - R(1.5) * usq);
            const R s0 = rq * R(12) * (R(1) - R(1.5) * vsq);
            f[0] = s0 + keep * (f[0] - e0);
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const R rw = rq * R(k36(i));
            R ep, em, sp, sm;
            feq_pair<R>(rw, cdot<R>(i, ux, uy, uz), usq, ep, em);
            feq_pair<R>(rw, cdot<R>(i, vx, vy, vz), vsq, sp, sm);
            f[i] = sp + keep * (f[i] - ep);
            f[i + 1] = sm + keep * (f[i + 1] - em);
        }
    } else {
        // second moment of f: sum_i c_ia c_ib f_i
        R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const R v = f[i];
            if (cx(i)) pxx += v;
            if (cy(i)) pyy += v;
            if (cz(i)) pzz += v;
            if (cx(i) && cy(i)) { if (cx(i) == cy(i)) pxy += v; else pxy -= v; }
            if (cx(i) && cz(i)) { if (cx(i) == cz(i)) pxz += v; else pxz -= v; }
            if (cy(i) && cz(i)) { if (cy(i) == cz(i)) pyz += v; else pyz -= v; }
        }
        const R T0 = R(1) / R(3);
        pxx -= rho * (T0 + ux * ux);
        pyy -= rho * (T0 + uy * uy);
        pzz -= rho * (T0 + uz * uz);
        pxy -= rho * ux * uy;
        pxz -= rho * ux * uz;
        pyz -= rho * uy * uz;
        const R t = (pxx + pyy + pzz) / R(3);
        Third<R> th;
        if (REG == 2) {
            th.zero();
#pragma unroll
            for (int i = 1; i < Q; ++i) th.add(i, f[i]);
            th.finish(rho, ux, uy, uz);
        }
        // f^neq_i = (k_i / 8) (c_i c_i : Pi - tr(Pi) / 3)
        {
            const R s0 = rq * R(12) * (R(1) - R(1.5) * vsq);
            f[0] = s0 + keep * (R(-1.5) * t);
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            R cc = R(0);
            if (cx(i)) cc += pxx;
            if (cy(i)) cc += pyy;
            if (cz(i)) cc += pzz;
            if (cx(i) && cy(i)) cc += (cx(i) == cy(i) ? R(2) : R(-2)) * pxy;
            if (cx(i) && cz(i)) cc += (cx(i) == cz(i) ? R(2) : R(-2)) * pxz;
            if (cy(i) && cz(i)) cc += (cy(i) == cz(i) ? R(2) : R(-2)) * pyz;
            const R fneq = R(k36(i)) * R(0.125) * (cc - t);   // same for i and opp(i)
            const R f3 = REG == 2 ? th.odd(i) : R(0);          // odd: -f3 for opp(i)
            R sp, sm;
            feq_pair<R>(rq * R(k36(i)), cdot<R>(i, vx, vy, vz), vsq, sp, sm);
            f[i] = sp + keep * (fneq + f3);
            f[i + 1] = sm + keep * (fneq - f3);
        }
    }
}

}  // namespace lbm
