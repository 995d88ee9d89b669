// Reverse-mode (adjoint) step of the two-component D3Q19 Shan-Chen update.
// The paper has no adjoint; this differentiates the forward step of
// Sec. 2 (Eqs. 1-7, 10-11, 13, with either reading of the forcing term) by hand.
//
// Notation: f^n = pre-collision populations at step n (the gathered values),
// lambda^n = dL/df^n.  One forward step is
//   f*(y) = C(f^n(y), S(y)),  S^b(y) = sum_k w_k c_k rho^b(y + c_k),
//   f^{n+1}_i(y + c_i) = f*_i(y)      (or f^{n+1}_opp(i)(y) at a wall),
// so one reverse step is
//   lambda^n_i(x) = lambda_loc^n_i(x) + D^n_b(x)    (b = component of i),
//   lambda_loc^n  = (dC/df)^T mu,   a^n_b(y) = (dC/dS^b)^T mu,
//   D^n_b(x)      = dL/drho^b(x) = sum_k w_k c_k . a^n_b(x - c_k)
//                   (+ mirror-wall terms),
//   mu_i(y)       = lambda^{n+1}_i(y + c_i)  (or lambda^{n+1}_opp(i)(y) at a wall).
// lambda itself is never stored: the reverse step gathers
// mu_i(y) = lambda_loc^{n+1}_i(y + c_i) + D^{n+1}_b(y + c_i) from the previous
// step's lambda_loc and the small field D^{n+1}.  Parameter sensitivities
// dL/dG^{ab} and dL/dtau_a are accumulated per block in FP64.
//
// Kernels: k_adj_seed (lambda_loc^N = dL/drho at the last step, D^N = 0),
// k_adj_D (D from a), k_adj_local (mu gather + local reverse pass),
// k_adj_rho0 (dL/drho_0 = sum_i w_i lambda^0_i for an initial state
// f^eq(rho_0, u = 0)).
//
// Kernel templates of the reverse step; adj::adj_step_t is instantiated per
// storage format in lbm_adjoint_<format>.cu (compiled in parallel), and
// lbm_adjoint.cu dispatches over the formats.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kThreadsA = 256;
// Launch shape of k_adj_local per arithmetic type: CTAs of `threads` (a
// power of two), `blocks` of them resident per SM.  FP32: 128 x 5 (20 warps
// per SM at 96 registers, a few spilled, measured faster than 16 warps at 128
// registers without spills: the kernel waits on loads); FP64: 256 x 2.
template <class R>
struct AdjLaunch {
    static constexpr int threads = sizeof(R) == 8 ? 256 : 128;
    static constexpr int blocks = sizeof(R) == 8 ? 2 : 5;
};

// A cell and its wrapped neighbour offsets.  Cell indices fit 32 bits (a
// lattice of 2^32 cells would need 650 GB of populations); element offsets
// into the 2 x 19 arrays are formed in 64 bits.
struct Nb {
    unsigned cell;
    unsigned xo[3], yo[3], zo[3];
    bool zlo, zhi;   // z - 1 (resp. z + 1) is a wall site
};

template <class R>
__device__ __forceinline__ void nb_at(const Phys<R> &p, unsigned x, unsigned y, unsigned z, Nb &n)
{
    const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, nz = (unsigned)p.nz;
    const unsigned plane = nx * ny;
    n.cell = z * plane + y * nx + x;
    n.xo[0] = x == 0 ? nx - 1 : x - 1;
    n.xo[1] = x;
    n.xo[2] = x == nx - 1 ? 0 : x + 1;
    n.yo[0] = (y == 0 ? ny - 1 : y - 1) * nx;
    n.yo[1] = y * nx;
    n.yo[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    n.zo[0] = (z == 0 ? nz - 1 : z - 1) * plane;
    n.zo[1] = z * plane;
    n.zo[2] = (z == nz - 1 ? 0 : z + 1) * plane;
    n.zlo = p.wall_z && z == 0;
    n.zhi = p.wall_z && z == nz - 1;
}

template <class R>
__device__ __forceinline__ void nb_of(const Phys<R> &p, unsigned cell, Nb &n)
{
    const unsigned nx = (unsigned)p.nx, plane = nx * (unsigned)p.ny;
    const unsigned z = cell / plane;
    const unsigned rem = cell - z * plane;
    const unsigned y = rem / nx;
    nb_at(p, rem - y * nx, y, z, n);
}

__device__ __forceinline__ unsigned at(const Nb &n, int dx, int dy, int dz)
{
    return n.zo[1 + dz] + n.yo[1 + dy] + n.xo[1 + dx];
}


// Local reverse pass of one component a at one cell, run by a pair of lanes
// (lane l: component 0, lane l ^ 16: component 1, same cell).  The two
// components are coupled only through the mixture momentum and density, whose
// sums and sensitivities the pair exchanges by shuffles; each lane holds its
// component's 19 populations and 19 incoming sensitivities
//   mu_i(y) = lambda^{n+1}_i(y + c_i) = lambda_loc^{n+1}_i(y + c_i) + D^{n+1}_a(y + c_i)
// (or lambda^{n+1}_opp(i)(y) at a wall), and writes lambda_loc^n_i(y) of its
// component and a^n_b(y) of the other component b = 1 - a.
template <int S, int REG, bool SIN, bool MASK, bool WZ, int FORCE>
__device__ __forceinline__ void adj_half(const typename Store<S>::T *__restrict__ f,
                                         const typename Store<S>::R *__restrict__ rho,
                                         const typename Store<S>::R *__restrict__ lam_next,
                                         const typename Store<S>::R *__restrict__ Dn,
                                         typename Store<S>::R *__restrict__ lam_loc, typename Store<S>::R *__restrict__ aout,
                                         const Phys<typename Store<S>::R> &p, const Nb &n, int a, bool store,
                                         typename Store<S>::R &par_g, typename Store<S>::R &par_t, unsigned lw)
{
    using R = typename Store<S>::R;
    const long long N = p.N;
    // z walls exist only in the WZ instances (periodic lattices test nothing)
    const bool zlo = WZ && n.zlo, zhi = WZ && n.zhi;
    // element offsets inside one component's 19 arrays fit 32 bits (19 N < 2^32,
    // checked on the host): one 32-bit multiply-add per access
    const unsigned N32 = (unsigned)N;
    const unsigned full = 0xffffffffu;
    // ---- forward recomputation ------------------------------------------
    R fa[Q];
    R rref = p.rho0;   // *_REL formats: the cell's own reference density of component a
    if constexpr (Store<S>::kRel) {
        const float2 rr = state_ref(f, p.ref_off)[n.cell];
        rref = a == 0 ? rr.x : rr.y;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // x - c_i behind a z wall or a solid site of a mask: the link bounces back
        const bool wall = (cz(i) == 1 && zlo) || (cz(i) == -1 && zhi) || (MASK && i != 0 && ((lw >> i) & 1u));
        const unsigned e = wall ? (unsigned)opp(i) * N32 + n.cell : (unsigned)i * N32 + at(n, -cx(i), -cy(i), -cz(i));
        fa[i] = Store<S>::load(f + a + 2 * (size_t)e, w<R>(i) * rref);
    }
    // ---- incoming sensitivities (issued with the population loads, so that
    //      both sets of gathers are in flight together) ----------------------
    R mu[Q];
    {
        const R *lam_a = lam_next + (size_t)a * Q * (size_t)N;
        const R *D_a = Dn + (size_t)a * (size_t)N;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && zlo) || (cz(i) == 1 && zhi) ||
                              (MASK && i != 0 && ((lw >> opp(i)) & 1u));   // y + c_i solid
            const unsigned cell = wall ? n.cell : at(n, cx(i), cy(i), cz(i));
            const unsigned d = wall ? (unsigned)opp(i) : (unsigned)i;
            mu[i] = lam_a[d * N32 + cell] + D_a[cell];
        }
    }
    R ra = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) ra += fa[i];
#pragma unroll
    for (int i = 1; i < Q; i += 2) {   // opposite pairs: f_i - f_opp(i) first
        const R d = fa[i] - fa[i + 1];
        if (cx(i) == 1) jx += d; else if (cx(i) == -1) jx -= d;
        if (cy(i) == 1) jy += d; else if (cy(i) == -1) jy -= d;
        if (cz(i) == 1) jz += d; else if (cz(i) == -1) jz -= d;
    }
    // mixture density and momentum: both lanes of the pair form the same sums
    const R rt = ra + __shfl_xor_sync(full, ra, 16);
    R u0 = (jx + __shfl_xor_sync(full, jx, 16)) / rt;
    R u1 = (jy + __shfl_xor_sync(full, jy, 16)) / rt;
    R u2 = (jz + __shfl_xor_sync(full, jz, 16)) / rt;
    // S^b of the other component b (Eq. 7; wall sites carry Eq. 13's rho'):
    // stored by the replayed forward step (SIN, rho = the sums [3 b + d][cell])
    // or formed from the densities
    const int b = 1 - a;
    R Sb0 = 0, Sb1 = 0, Sb2 = 0;
    if (SIN) {
        Sb0 = rho[(long long)(3 * b + 0) * N + n.cell];
        Sb1 = rho[(long long)(3 * b + 1) * N + n.cell];
        Sb2 = rho[(long long)(3 * b + 2) * N + n.cell];
    } else {
        const R *rbp = rho + (long long)b * N;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && zlo) || (cz(i) == 1 && zhi);
            R rv;
            if (wall) {
                rv = p.rho_s[b];
                if (p.wall_mirror) rv += rbp[at(n, cx(i), cy(i), 0)];
            } else {
                rv = rbp[at(n, cx(i), cy(i), cz(i))];
            }
            const R wr = w<R>(i) * rv;
            if (cx(i) == 1) Sb0 += wr; else if (cx(i) == -1) Sb0 -= wr;
            if (cy(i) == 1) Sb1 += wr; else if (cy(i) == -1) Sb1 -= wr;
            if (cz(i) == 1) Sb2 += wr; else if (cz(i) == -1) Sb2 -= wr;
        }
    }
    const R Ga = a == 0 ? p.G12 : p.G21;
    const R ga0 = Ga * Sb0 + p.gext[0], ga1 = Ga * Sb1 + p.gext[1], ga2 = Ga * Sb2 + p.gext[2];   // g^a
    // Guo's forcing (R2b): both components relax toward f^eq at the common
    // u* = u + (F^1 + F^2) / (2 rho), F^a = rho^a g^a; from here on u stands
    // for u* and v = u* (the exact-difference formulas below then hold with
    // v = u, and the forcing term's derivatives are added)
    R F0 = 0, F1 = 0, F2 = 0;
    if constexpr (FORCE == FORCE_GUO) {
        F0 = ra * ga0; F1 = ra * ga1; F2 = ra * ga2;
        const R h = R(0.5) / rt;
        u0 += (F0 + __shfl_xor_sync(full, F0, 16)) * h;
        u1 += (F1 + __shfl_xor_sync(full, F1, 16)) * h;
        u2 += (F2 + __shfl_xor_sync(full, F2, 16)) * h;
    }
    const R usq = u0 * u0 + u1 * u1 + u2 * u2;
    const bool guo = FORCE == FORCE_GUO;
    const R v0 = guo ? u0 : u0 + ga0, v1 = guo ? u1 : u1 + ga1, v2 = guo ? u2 : u2 + ga2;
    const R vsq = v0 * v0 + v1 * v1 + v2 * v2;
    const R omega = a == 0 ? p.omega[0] : p.omega[1];
    const R keep = R(1) - omega;
    const R rq = ra / R(36);
    // regularized: Pi = sum c c f - rho (T0 I + u u), as xx, yy, zz, xy, xz, yz
    R Pi[6] = {0, 0, 0, 0, 0, 0}, tr = 0;
    if (REG) {
        const R T0 = R(1) / R(3);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (cx(i)) Pi[0] += fa[i];
            if (cy(i)) Pi[1] += fa[i];
            if (cz(i)) Pi[2] += fa[i];
            if (cx(i) && cy(i)) Pi[3] += R(cx(i) * cy(i)) * fa[i];
            if (cx(i) && cz(i)) Pi[4] += R(cx(i) * cz(i)) * fa[i];
            if (cy(i) && cz(i)) Pi[5] += R(cy(i) * cz(i)) * fa[i];
        }
        Pi[0] -= ra * (T0 + u0 * u0);
        Pi[1] -= ra * (T0 + u1 * u1);
        Pi[2] -= ra * (T0 + u2 * u2);
        Pi[3] -= ra * u0 * u1;
        Pi[4] -= ra * u0 * u2;
        Pi[5] -= ra * u1 * u2;
        if constexpr (FORCE == FORCE_GUO) {   // Pi of f - f^eq(u*) + F/2: + (u* F + F u*) / 2
            Pi[0] += u0 * F0; Pi[1] += u1 * F1; Pi[2] += u2 * F2;
            Pi[3] += R(0.5) * (u0 * F1 + u1 * F0);
            Pi[4] += R(0.5) * (u0 * F2 + u2 * F0);
            Pi[5] += R(0.5) * (u1 * F2 + u2 * F1);
        }
        tr = Pi[0] + Pi[1] + Pi[2];
    }
    // third-order part (REG = 2): S_a, D_a of struct Third for this component
    Third<R> th;
    if (REG == 2) {
        th.zero();
#pragma unroll
        for (int i = 1; i < Q; ++i) th.add(i, fa[i]);
        th.finish(ra, u0, u1, u2);
    }
    // ---- reverse pass -------------------------------------------------------
    // BGK:         f* = E(rho, v) + keep (f - E(rho, u))
    // regularized: f* = E(rho, v) + keep (k_i / 8) (c c : Pi - tr(Pi) / 3)
    // with E_i(rho, x) = (rho / 36) k_i P(c_i . x, x . x)
    // Opposite directions (i, i + 1) share k_i and |c_i . x|: with s = k (mu_i +
    // mu_opp), d = k (mu_i - mu_opp) and P(+-c) = E +- O, grad P(+-c) = A +- B,
    // the pair contributes E s + O d to the density sensitivity and (A d + B s)
    // c_i to the velocity one.
    R Kbar = 0, rbar = 0;
    R vbx = 0, vby = 0, vbz = 0, vbv = 0, ubx = 0, uby = 0, ubz = 0, ubv = 0;
    R pb[6] = {0, 0, 0, 0, 0, 0};
    R sb[3] = {0, 0, 0}, db[3] = {0, 0, 0};   // dL/dS_a, dL/dD_a (REG = 2)
    // Guo forcing term T_i = (k_i / 36) (9 (c.u*) (c.F) - 3 u*.F + 3 c.F), times cf:
    // 36 sum mu T, and 36 x its gradients in u* (Tu - 3 F sgs) and F (TF - 3 u* sgs)
    const R uF = u0 * F0 + u1 * F1 + u2 * F2;
    R Tsum = 0, sgs = 0, Tux = 0, Tuy = 0, Tuz = 0, TFx = 0, TFy = 0, TFz = 0;
    {
        // rest population: c = 0, k = 12
        const R m = mu[0], mk = m * R(12);
        if constexpr (FORCE == FORCE_GUO) {
            Tsum += mk * (R(-3) * uF);
            sgs += mk;
        }
        rbar += mk * (R(1) - R(1.5) * vsq);
        vbv += R(3) * mk;
        if (!REG) {
            const R Pu = R(1) - R(1.5) * usq;
            Kbar += m * (fa[0] - rq * R(12) * Pu);
            rbar -= keep * mk * Pu;
            ubv += R(3) * mk;
        } else {
            Kbar += mk * R(0.125) * (-tr / R(3));
            const R nb = keep * mk * R(0.125);
            pb[0] -= nb / R(3);
            pb[1] -= nb / R(3);
            pb[2] -= nb / R(3);
        }
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const R ki = R(k36(i));
        const R sg = (mu[i] + mu[i + 1]) * ki, df = (mu[i] - mu[i + 1]) * ki;
        const R cv = cdot<R>(i, v0, v1, v2), cv2 = cv * cv;
        const R E = R(1) + R(4.5) * cv2 - R(1.5) * vsq, O = cv * (R(3) + R(4.5) * cv2 - R(4.5) * vsq);
        rbar += E * sg + O * df;
        if constexpr (FORCE == FORCE_GUO) {
            const R cu = cdot<R>(i, u0, u1, u2), cF = cdot<R>(i, F0, F1, F2);
            Tsum += sg * (R(9) * cu * cF - R(3) * uF) + R(3) * df * cF;
            sgs += sg;
            const R tu = R(9) * sg * cF, tF = R(9) * sg * cu + R(3) * df;
            if (cx(i)) { Tux += R(cx(i)) * tu; TFx += R(cx(i)) * tF; }
            if (cy(i)) { Tuy += R(cy(i)) * tu; TFy += R(cy(i)) * tF; }
            if (cz(i)) { Tuz += R(cz(i)) * tu; TFz += R(cz(i)) * tF; }
        }
        const R t = (R(3) + R(13.5) * cv2 - R(4.5) * vsq) * df + R(9) * cv * sg;
        if (cx(i)) vbx += R(cx(i)) * t;
        if (cy(i)) vby += R(cy(i)) * t;
        if (cz(i)) vbz += R(cz(i)) * t;
        vbv += R(3) * sg + R(9) * cv * df;
        if (!REG) {
            const R cu = cdot<R>(i, u0, u1, u2), cu2 = cu * cu;
            const R Eu = R(1) + R(4.5) * cu2 - R(1.5) * usq, Ou = cu * (R(3) + R(4.5) * cu2 - R(4.5) * usq);
            const R Pm = Eu * sg + Ou * df;
            Kbar += mu[i] * fa[i] + mu[i + 1] * fa[i + 1] - rq * Pm;
            rbar -= keep * Pm;
            const R tu = (R(3) + R(13.5) * cu2 - R(4.5) * usq) * df + R(9) * cu * sg;
            if (cx(i)) ubx += R(cx(i)) * tu;
            if (cy(i)) uby += R(cy(i)) * tu;
            if (cz(i)) ubz += R(cz(i)) * tu;
            ubv += R(3) * sg + R(9) * cu * df;
        } else {
            const int c0 = cx(i), c1 = cy(i), c2 = cz(i);
            const R ccP = R(c0 * c0) * Pi[0] + R(c1 * c1) * Pi[1] + R(c2 * c2) * Pi[2] + R(2 * c0 * c1) * Pi[3] +
                          R(2 * c0 * c2) * Pi[4] + R(2 * c1 * c2) * Pi[5];
            Kbar += sg * R(0.125) * (ccP - tr / R(3));
            const R nb = keep * sg * R(0.125);
            pb[0] += nb * (R(c0 * c0) - R(1) / R(3));
            pb[1] += nb * (R(c1 * c1) - R(1) / R(3));
            pb[2] += nb * (R(c2 * c2) - R(1) / R(3));
            if (c0 && c1) pb[3] += nb * R(c0 * c1);
            if (c0 && c2) pb[4] += nb * R(c0 * c2);
            if (c1 && c2) pb[5] += nb * R(c1 * c2);
            if (REG == 2) {
                // f*_i +- keep (k_i / 8) sum_a (S_a h3s3(i, a) + D_a h3d(i, a)) for i, opp(i)
                Kbar += df * R(0.125) * (th.odd(i) / (R(k36(i)) * R(0.125)));
                const R nd = keep * df * R(0.125);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (h3s3(i, q)) sb[q] += nd * R(h3s3(i, q));
                    if (h3d(i, q)) db[q] += nd * R(h3d(i, q));
                }
            }
        }
    }
    rbar /= R(36);
    // dL/dv^a
    const R vbar0 = rq * (vbx - v0 * vbv), vbar1 = rq * (vby - v1 * vbv), vbar2 = rq * (vbz - v2 * vbv);
    R ub0 = vbar0, ub1 = vbar1, ub2 = vbar2;
    if (!REG) {
        ub0 -= keep * rq * (ubx - u0 * ubv);
        ub1 -= keep * rq * (uby - u1 * ubv);
        ub2 -= keep * rq * (ubz - u2 * ubv);
    } else {
        // pb holds dL/dPi for xx, yy, zz and one of each symmetric off-diagonal pair
        const R T0 = R(1) / R(3);
        rbar -= pb[0] * (T0 + u0 * u0) + pb[1] * (T0 + u1 * u1) + pb[2] * (T0 + u2 * u2) +
                R(2) * (pb[3] * u0 * u1 + pb[4] * u0 * u2 + pb[5] * u1 * u2);
        ub0 -= R(2) * ra * (pb[0] * u0 + pb[3] * u1 + pb[4] * u2);
        ub1 -= R(2) * ra * (pb[3] * u0 + pb[1] * u1 + pb[5] * u2);
        ub2 -= R(2) * ra * (pb[4] * u0 + pb[5] * u1 + pb[2] * u2);
        if (REG == 2) {
            // S_a = (1/3) sum h3s3 f - rho u_a (u_b^2 + u_c^2) / 2,
            // D_a = sum h3d f - 3/2 rho u_a (u_b^2 - u_c^2)   (b < c the other axes)
            const R u[3] = {u0, u1, u2};
            R ubq[3] = {0, 0, 0};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int qb = q == 0 ? 1 : 0, qc = q == 2 ? 1 : 2;
                const R ua = u[q], ubb = u[qb], ucc = u[qc];
                rbar -= sb[q] * R(0.5) * ua * (ubb * ubb + ucc * ucc) + db[q] * R(1.5) * ua * (ubb * ubb - ucc * ucc);
                ubq[q] -= ra * (sb[q] * R(0.5) * (ubb * ubb + ucc * ucc) + db[q] * R(1.5) * (ubb * ubb - ucc * ucc));
                ubq[qb] -= ra * ua * ubb * (sb[q] + R(3) * db[q]);
                ubq[qc] -= ra * ua * ucc * (sb[q] - R(3) * db[q]);
            }
            ub0 += ubq[0];
            ub1 += ubq[1];
            ub2 += ubq[2];
        }
    }
    // Guo: the forcing term's u* and F^a derivatives (and, regularized, those of
    // the (u* F + F u*) / 2 part of Pi); dL/dF^a collects them
    R Fb0 = 0, Fb1 = 0, Fb2 = 0;
    if constexpr (FORCE == FORCE_GUO) {
        const R cf = (REG ? R(0.5) : R(1) - R(0.5) * omega) / R(36);
        ub0 += cf * (Tux - R(3) * F0 * sgs);
        ub1 += cf * (Tuy - R(3) * F1 * sgs);
        ub2 += cf * (Tuz - R(3) * F2 * sgs);
        Fb0 = cf * (TFx - R(3) * u0 * sgs);
        Fb1 = cf * (TFy - R(3) * u1 * sgs);
        Fb2 = cf * (TFz - R(3) * u2 * sgs);
        if (REG) {
            ub0 += pb[0] * F0 + pb[3] * F1 + pb[4] * F2;
            ub1 += pb[3] * F0 + pb[1] * F1 + pb[5] * F2;
            ub2 += pb[4] * F0 + pb[5] * F1 + pb[2] * F2;
            Fb0 += pb[0] * u0 + pb[3] * u1 + pb[4] * u2;
            Fb1 += pb[3] * u0 + pb[1] * u1 + pb[5] * u2;
            Fb2 += pb[4] * u0 + pb[5] * u1 + pb[2] * u2;
        } else {
            Kbar += Tsum / R(72);   // cf = 1 - omega / 2 = (1 + keep) / 2
        }
    }
    // u = j / rho over both components: dL/dj = ubar / rho, dL/drho += -(ubar . u) / rho
    // (Guo: u* = j / rho + (F^1 + F^2) / (2 rho) gives the same with u*, and
    // dL/dF^a += ubar / (2 rho))
    const R U0 = ub0 + __shfl_xor_sync(full, ub0, 16);
    const R U1 = ub1 + __shfl_xor_sync(full, ub1, 16);
    const R U2 = ub2 + __shfl_xor_sync(full, ub2, 16);
    const R jb0 = U0 / rt, jb1 = U1 / rt, jb2 = U2 / rt;
    if constexpr (FORCE == FORCE_GUO) {
        const R h = R(0.5) / rt;
        Fb0 += U0 * h; Fb1 += U1 * h; Fb2 += U2 * h;
        rbar += Fb0 * ga0 + Fb1 * ga1 + Fb2 * ga2;   // F^a = rho^a g^a
    }
    const R base = rbar - (U0 * u0 + U1 * u1 + U2 * u2) / rt;
    // dL/dg^a: the velocity shift v = u + g^a (exact difference), or rho^a dL/dF^a (Guo)
    const R gb0 = guo ? ra * Fb0 : vbar0, gb1 = guo ? ra * Fb1 : vbar1, gb2 = guo ? ra * Fb2 : vbar2;
    if (store && MASK && (lw & 1u)) {
        // solid site: no populations, no sensitivities (a = 0 keeps it out of D)
        R *lo = lam_loc + (size_t)a * Q * (size_t)N + n.cell;
#pragma unroll
        for (int i = 0; i < Q; ++i) lo[(unsigned)i * N32] = R(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) aout[((long long)b * 3 + d) * N + n.cell] = R(0);
    } else if (store) {
        R *lo = lam_loc + (size_t)a * Q * (size_t)N + n.cell;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            R l = base + cdot<R>(i, jb0, jb1, jb2);
            if (!REG) {
                l += keep * mu[i];
            } else {
                const int c0 = cx(i), c1 = cy(i), c2 = cz(i);
                l += R(c0 * c0) * pb[0] + R(c1 * c1) * pb[1] + R(c2 * c2) * pb[2] + R(2 * c0 * c1) * pb[3] +
                     R(2 * c0 * c2) * pb[4] + R(2 * c1 * c2) * pb[5];
                if (REG == 2) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (h3s3(i, q)) l += sb[q] * (R(h3s3(i, q)) / R(3));
                        if (h3d(i, q)) l += db[q] * R(h3d(i, q));
                    }
                }
            }
            lo[(unsigned)i * N32] = l;
        }
        // g^a = G^{ab} S^b + g_ext:  dL/dS^b = G^{ab} dL/dg^a,  dL/dG^{ab} = dL/dg^a . S^b
        aout[((long long)b * 3 + 0) * N + n.cell] = Ga * gb0;
        aout[((long long)b * 3 + 1) * N + n.cell] = Ga * gb1;
        aout[((long long)b * 3 + 2) * N + n.cell] = Ga * gb2;
        par_g += gb0 * Sb0 + gb1 * Sb1 + gb2 * Sb2;
        // keep = 1 - 1/tau: dkeep/dtau = 1/tau^2
        par_t += Kbar * omega * omega;
    }
}

// Grid-stride over groups of 16 cells per warp; lanes 0-15 take component 0
// and lanes 16-31 component 1 of the same 16 cells.  Per-block FP64 partials
// of dL/dG^{12}, dL/dG^{21}, dL/dtau_1, dL/dtau_2 accumulate over the steps.
// MASK: links holds the mask's link words (bit 0: solid site; bit i: x - c_i
// solid).  The lanes of a solid site still run the arithmetic (on meaningless
// values), so that both lanes of every pair take part in the shuffles, and
// store zeros.
template <int S, int REG, bool SIN, bool MASK, bool WZ, int FORCE>
__global__ void __launch_bounds__(AdjLaunch<typename Store<S>::R>::threads, AdjLaunch<typename Store<S>::R>::blocks)
k_adj_local(const typename Store<S>::T *__restrict__ f, const typename Store<S>::R *__restrict__ rho,
            const typename Store<S>::R *__restrict__ lam_next, const typename Store<S>::R *__restrict__ Dn,
            typename Store<S>::R *__restrict__ lam_loc, typename Store<S>::R *__restrict__ aout,
            double *__restrict__ partials, Phys<typename Store<S>::R> p, const unsigned *__restrict__ links)
{
    constexpr int kThreadsL = AdjLaunch<typename Store<S>::R>::threads;
    const int lane = threadIdx.x & 31;
    const int a = lane >> 4;
    const long long warps = (long long)gridDim.x * (kThreadsL / 32);
    const long long groups = (p.N + 15) / 16;
    // per-thread partials in the arithmetic type over the thread's cells (a few
    // tens per step), summed in FP64 across the block: the FP64 pipe is a
    // small fraction of the FP32 one on this GPU
    typename Store<S>::R pg = 0, pt = 0;
    // the lane's cell advances by the fixed stride 16 warps per iteration: its
    // coordinates advance by the stride's (sx, sy, sz) with carries, so the
    // loop divides by the lattice sizes only once
    // (19 N < 2^32, checked on the host, so cells, strides and z fit 32 bits)
    const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, plane = nx * ny;
    const unsigned stride = (unsigned)warps * 16u;
    const unsigned sx = stride % nx, sy = (stride / nx) % ny, sz = stride / plane;
    const long long wg0 = (long long)blockIdx.x * (kThreadsL / 32) + (threadIdx.x >> 5);
    const unsigned c0 = (unsigned)wg0 * 16u + (unsigned)(lane & 15);
    unsigned px = c0 % nx, py = (c0 / nx) % ny, pz = c0 / plane;
    for (long long wg = wg0; wg < groups; wg += warps) {
        const long long c = wg * 16 + (lane & 15);
        const bool valid = c < p.N;
        Nb n;
        if (valid) nb_at(p, px, py, pz, n);
        else nb_at(p, nx - 1, ny - 1, (unsigned)(p.nz - 1), n);
        px += sx;
        const unsigned cxr = px >= nx ? 1u : 0u;
        px -= cxr * nx;
        py += sy + cxr;
        const unsigned cyr = py >= ny ? 1u : 0u;
        py -= cyr * ny;
        pz += sz + cyr;
        const unsigned lw = MASK ? __ldg(links + n.cell) : 0u;
        adj_half<S, REG, SIN, MASK, WZ, FORCE>(f, rho, lam_next, Dn, lam_loc, aout, p, n, a, valid, pg, pt, lw);
    }
    // lanes of component a hold parts of par[a] and par[2 + a]
    __shared__ double sh[4][kThreadsL];
    const int t = threadIdx.x;
    for (int k = 0; k < 4; ++k) sh[k][t] = 0;
    sh[a][t] = pg;
    sh[2 + a][t] = pt;
    __syncthreads();
    for (int s = kThreadsL / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int k = 0; k < 4; ++k) sh[k][t] += sh[k][t + s];
        __syncthreads();
    }
    if (t < 4) partials[(long long)blockIdx.x * 4 + t] += sh[t][0];
}

// D_b(x) = dL/drho^b(x) = sum_k w_k c_k . a_b(x - c_k), plus the mirror-wall
// terms: a wall site y + c_k seen from y presents the density of its mirror
// cell y + (c_kx, c_ky, 0).
//
// Output tiles of 32 x 8 x DZ cells: the six fields a_b,d over the tile and a
// one-cell margin (periodic images in x and y; in z periodic images, or zeros
// for wall sites, whose terms the sum leaves out) are staged in shared memory
// with coalesced loads, then each thread sums its z column of DZ cells from
// shared memory, plane by plane (below).
constexpr int kDX = 32, kDY = 8;
template <class R>
struct DTile {
    static constexpr int DZ = sizeof(R) == 8 ? 4 : 8;   // 98 KB (FP64) / 82 KB (FP32) of staging
    static constexpr int BX = kDX + 2, BY = kDY + 2, BZ = DZ + 2;
    static constexpr int BOX = BX * BY * BZ;
    static constexpr size_t kSmem = sizeof(R) * 6 * (size_t)BOX;
};

template <class R>
__global__ void __launch_bounds__(kThreadsA, 2)
k_adj_D(const R *__restrict__ a, R *__restrict__ D, Phys<R> p, int ntx)
{
    using T = DTile<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *box = reinterpret_cast<R *>(smem_raw);   // [6][BZ][BY][BX]
    // wrapped offsets of the box's rows (hz, hy) and columns hx, formed once per
    // CTA (a row behind a z wall is marked -1 and staged as zeros)
    __shared__ int row_off[T::BZ * T::BY];
    __shared__ int col_off[T::BX];
    const int t = threadIdx.x;
    const int x0 = (blockIdx.x % ntx) * kDX, y0 = (blockIdx.x / ntx) * kDY, z0 = blockIdx.y * T::DZ;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const unsigned N32 = (unsigned)p.N;   // 6 N < 2^32 (19 N is, on the host)
    if (t < T::BZ * T::BY) {
        const int hy = t % T::BY, hz = t / T::BY;
        int gy = (y0 - 1 + hy) % ny;
        if (gy < 0) gy += ny;
        int gz = z0 - 1 + hz;
        bool inside = true;
        if (p.wall_z) {
            inside = gz >= 0 && gz < nz;
        } else {
            gz %= nz;
            if (gz < 0) gz += nz;
        }
        row_off[t] = inside ? (gz * ny + gy) * nx : -1;
    } else if (t - T::BZ * T::BY < T::BX) {
        const int hx = t - T::BZ * T::BY;
        int gx = (x0 - 1 + hx) % nx;
        if (gx < 0) gx += nx;
        col_off[hx] = gx;
    }
    static_assert(T::BZ * T::BY + T::BX <= kThreadsA, "one offset per thread");
    __syncthreads();
    // all of the thread's loads are issued before the first shared-memory
    // store, so that they are in flight together
    constexpr int kIt = (T::BOX + kThreadsA - 1) / kThreadsA;
    R val[kIt][6];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int h = it * kThreadsA + t;
        const int ro = h < T::BOX ? row_off[h / T::BX] : -1;
        const unsigned c = ro >= 0 ? (unsigned)(ro + col_off[h % T::BX]) : 0u;
#pragma unroll
        for (int q = 0; q < 6; ++q) val[it][q] = ro >= 0 ? __ldg(a + (unsigned)q * N32 + c) : R(0);
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
        const int h = it * kThreadsA + t;
        if (h < T::BOX) {
#pragma unroll
            for (int q = 0; q < 6; ++q) box[q * T::BOX + h] = val[it][q];
        }
    }
    __syncthreads();
    const int lx = t % kDX, ly = t / kDX;
    const int x = x0 + lx, y = y0 + ly;
    if (x >= nx || y >= ny) return;
    // Sweep over the box planes P = 0 .. DZ + 1.  Grouped by source plane, the
    // 18 links of D at a cell split into the 8 links within its plane (in),
    // the 5 from the plane below (lo: c_z = +1) and the 5 from the plane above
    // (hi: c_z = -1); each needs only these 17 values of a source plane
    // (offsets (dx, dy) from the cell's column):
    //   a_x at (-+1, 0), (-+1, -+1);  a_y at (0, -+1), (-+1, -+1);
    //   a_z at (0, 0), (-+1, 0), (0, -+1),
    // with  A = a_x(-1,0) - a_x(1,0) + a_y(0,-1) - a_y(0,1),
    //       Zs = a_z(-1,0) + a_z(1,0) + a_z(0,-1) + a_z(0,1):
    //   in = A / 18 + [a_x(-1,-1) + a_y(-1,-1) - a_x(1,1) - a_y(1,1)
    //                  + a_x(-1,1) - a_y(-1,1) - a_x(1,-1) + a_y(1,-1)] / 36,
    //   lo =  a_z(0,0) / 18 + (A + Zs) / 36,   hi = -a_z(0,0) / 18 + (A - Zs) / 36.
    // Plane P is the lower plane of cell P, the own plane of cell P - 1 and
    // the upper plane of cell P - 2, so each plane's values are read once.
    // The mirror terms of a cell next to a z wall are the links that would
    // come through the wall, evaluated in its own plane: hi at z = 0, lo at
    // z = nz - 1.
    const R r18 = R(1) / R(18), r36 = R(1) / R(36);
    R acc[T::DZ][2];
#pragma unroll
    for (int k = 0; k < T::DZ; ++k) acc[k][0] = acc[k][1] = R(0);
#pragma unroll
    for (int P = 0; P < T::DZ + 2; ++P) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const R *bx = box + (3 * b + 0) * T::BOX + (P * T::BY + ly + 1) * T::BX + lx + 1;
            const R *by = bx + T::BOX, *bz = bx + 2 * T::BOX;
            auto o = [](int dx, int dy) { return dy * T::BX + dx; };
            const R A = bx[o(-1, 0)] - bx[o(1, 0)] + by[o(0, -1)] - by[o(0, 1)];
            const R Zc = bz[o(0, 0)];
            const R Zs = bz[o(-1, 0)] + bz[o(1, 0)] + bz[o(0, -1)] + bz[o(0, 1)];
            const R lo = Zc * r18 + (A + Zs) * r36;
            const R hi = (A - Zs) * r36 - Zc * r18;
            if (P < T::DZ) acc[P][b] += lo;
            if (P >= 1 && P - 1 < T::DZ) {
                const R E = bx[o(-1, -1)] + by[o(-1, -1)] - bx[o(1, 1)] - by[o(1, 1)] + bx[o(-1, 1)] -
                            by[o(-1, 1)] - bx[o(1, -1)] + by[o(1, -1)];
                acc[P - 1][b] += A * r18 + E * r36;
                if (p.wall_z && p.wall_mirror) {
                    const int z = z0 + P - 1;
                    if (z == 0) acc[P - 1][b] += hi;
                    if (z == nz - 1) acc[P - 1][b] += lo;
                }
            }
            if (P >= 2) acc[P - 2][b] += hi;
        }
    }
#pragma unroll
    for (int k = 0; k < T::DZ; ++k) {
        const int z = z0 + k;
        if (z < nz) {
            const unsigned cell = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
            D[cell] = acc[k][0];
            D[N32 + cell] = acc[k][1];
        }
    }
}

// Mirror wall model under a mask: a solid site s presents
// rho_w(s) = sum_j k_j rho(s + c_j) / sum_j k_j + rho_s over its fluid
// neighbours s + c_j (Eq. 13, modified model), so each fluid cell x next to s
// gains dL/drho_w(s) k_j / sum_j k_j.  dL/drho_w(s) is the regular D sum at s
// (k_adj_D, with a = 0 at solid sites), which this pass reads and leaves as
// it is; it runs over the fluid cells with a solid neighbour.
template <class R>
__global__ void __launch_bounds__(kThreadsA)
k_adj_D_wall(R *__restrict__ D, const unsigned char *__restrict__ solid, Phys<R> p,
             const unsigned *__restrict__ cells, long long n)
{
    const long long t = (long long)blockIdx.x * kThreadsA + threadIdx.x;
    if (t >= n) return;
    Nb nx_;
    nb_of(p, cells[t], nx_);
    const unsigned N32 = (unsigned)p.N;
    R add0 = 0, add1 = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const unsigned sc = at(nx_, cx(i), cy(i), cz(i));
        if (!__ldg(solid + sc)) continue;
        Nb ns;
        nb_of(p, sc, ns);
        int den36 = 0;
#pragma unroll
        for (int j = 1; j < Q; ++j)
            if (!__ldg(solid + at(ns, cx(j), cy(j), cz(j)))) den36 += k36(j);
        const R wgt = R(k36(i)) / R(den36);
        add0 += wgt * D[sc];
        add1 += wgt * D[N32 + sc];
    }
    D[nx_.cell] += add0;
    D[N32 + nx_.cell] += add1;
}

template <class R, class G>
__global__ void __launch_bounds__(kThreadsA)
k_adj_seed(const G *__restrict__ g1, const G *__restrict__ g2, R *__restrict__ lam, long long N)
{
    const long long c = (long long)blockIdx.x * kThreadsA + threadIdx.x;
    if (c >= N) return;
    const R v1 = g1 ? (R)g1[c] : R(0);
    const R v2 = g2 ? (R)g2[c] : R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        lam[(long long)i * N + c] = v1;
        lam[(long long)(Q + i) * N + c] = v2;
    }
}

// dL/drho^a_0 = sum_i w_i lambda^0_i = sum_i w_i lambda_loc^0_i + D^0_a (sum_i w_i = 1).
template <class R>
__global__ void __launch_bounds__(kThreadsA)
k_adj_rho0(const R *__restrict__ lam, const R *__restrict__ D, double *__restrict__ g1, double *__restrict__ g2,
           long long N, const unsigned char *__restrict__ solid)
{
    const long long c = (long long)blockIdx.x * kThreadsA + threadIdx.x;
    if (c >= N) return;
    if (solid && solid[c]) {   // a solid site holds no fluid: its initial density does not enter
        if (g1) g1[c] = 0.0;
        if (g2) g2[c] = 0.0;
        return;
    }
    double s1 = 0, s2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s1 += wd(i) * (double)lam[(long long)i * N + c];
        s2 += wd(i) * (double)lam[(long long)(Q + i) * N + c];
    }
    if (g1) g1[c] = s1 + (double)D[c];
    if (g2) g2[c] = s2 + (double)D[N + c];
}

template <class R>
Phys<R> make_phys_a(const HostPhys &h)
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

inline unsigned gridA(long long N) { return (unsigned)((N + kThreadsA - 1) / kThreadsA); }

constexpr int kMaxAttrDevices = 64;

// Launch of the tiled D pass; its dynamic shared-memory attribute belongs to
// the device context and is set once per device.
template <class R>
cudaError_t launch_adj_D(const HostPhys &h, const R *a, R *D, const Phys<R> &p, cudaStream_t s)
{
    using T = DTile<R>;
    const int ntx = (h.nx + kDX - 1) / kDX, nty = (h.ny + kDY - 1) / kDY;
    const long long zb = (h.nz + T::DZ - 1) / T::DZ;
    if ((long long)ntx * nty >= (1LL << 31) || zb > 65535) return cudaErrorInvalidConfiguration;
    static std::atomic<int> attr_set[kMaxAttrDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kMaxAttrDevices;
    if (!cached || !attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute((const void *)k_adj_D<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::kSmem);
        if (e != cudaSuccess) return e;
        if (cached) attr_set[dev].store(1, std::memory_order_release);
    }
    k_adj_D<R><<<dim3((unsigned)(ntx * nty), (unsigned)zb), kThreadsA, T::kSmem, s>>>(a, D, p, ntx);
    return cudaGetLastError();
}

}  // namespace

namespace adj {

template <int S>
cudaError_t adj_step_t(const HostPhys &h, const void *f, const void *rho, int rho_is_sums, const void *lam_next,
                       const void *Dn, void *lam_loc, void *a, void *Dout, double *partials, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const Phys<R> p = make_phys_a<R>(h);
#define LBM_ADJ(REG_, SIN_, MASK_, WZ_)                                                                           \
    do {                                                                                                          \
        if (h.forcing == FORCE_GUO)                                                                               \
            k_adj_local<S, REG_, SIN_, MASK_, WZ_, FORCE_GUO><<<nblk, AdjLaunch<R>::threads, 0, s>>>(             \
                (const T *)f, (const R *)rho, (const R *)lam_next, (const R *)Dn, (R *)lam_loc, (R *)a, partials, \
                p, h.links);                                                                                      \
        else                                                                                                      \
            k_adj_local<S, REG_, SIN_, MASK_, WZ_, FORCE_EDM><<<nblk, AdjLaunch<R>::threads, 0, s>>>(             \
                (const T *)f, (const R *)rho, (const R *)lam_next, (const R *)Dn, (R *)lam_loc, (R *)a, partials, \
                p, h.links);                                                                                      \
    } while (0)
#define LBM_ADJ_REG(SIN_, MASK_, WZ_)                  \
    do {                                               \
        if (reg == 1) LBM_ADJ(1, SIN_, MASK_, WZ_);    \
        else if (reg == 2) LBM_ADJ(2, SIN_, MASK_, WZ_); \
        else LBM_ADJ(0, SIN_, MASK_, WZ_);             \
    } while (0)
    const int reg = h.collision == LBM_REGULARIZED ? 1 : (h.collision == LBM_REGULARIZED3 ? 2 : 0);
    const int nblk = adjoint_blocks(h.storage);
    // geometry instances: a mask (periodic z), z walls, or periodic
    if (h.links) {
        if (rho_is_sums) LBM_ADJ_REG(true, true, false);
        else LBM_ADJ_REG(false, true, false);
    } else if (h.wall_z) {
        if (rho_is_sums) LBM_ADJ_REG(true, false, true);
        else LBM_ADJ_REG(false, false, true);
    } else {
        if (rho_is_sums) LBM_ADJ_REG(true, false, false);
        else LBM_ADJ_REG(false, false, false);
    }
#undef LBM_ADJ_REG
#undef LBM_ADJ
    cudaError_t e = launch_adj_D<R>(h, (const R *)a, (R *)Dout, p, s);
    if (e == cudaSuccess && h.links && h.wall_mirror && h.n_bfluid > 0) {
        k_adj_D_wall<R><<<gridA(h.n_bfluid), kThreadsA, 0, s>>>((R *)Dout, h.solid, p, h.bfluid, h.n_bfluid);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace adj
}  // namespace lbm
