// Reverse-mode (adjoint) step of the two-component D3Q19 Shan-Chen update.
// The paper has no adjoint; this differentiates the forward step of
// Sec. 2 (Eqs. 1-7, 10-11, 13 with the exact-difference forcing) by hand.
//
// Notation: f^n = pre-collision populations at step n (the gathered values),
// lambda^n = dL/df^n.  One forward step is
//   f*(y) = C(f^n(y), S(y)),  S^b(y) = sum_k w_k c_k rho^b(y + c_k),
//   f^{n+1}_i(y + c_i) = f*_i(y)      (or f^{n+1}_opp(i)(y) at a wall),
// so one reverse step is
//   mu_i(y)      = lambda^{n+1}_i(y + c_i)   (or lambda^{n+1}_opp(i)(y) at a wall)
//   lambda_loc   = (dC/df)^T mu,   a^b(y) = (dC/dS^b)^T mu
//   lambda^n_i(x) = lambda_loc_i(x) + D^b(x),   D^b(x) = dL/drho^b(x)
//                 = sum_k w_k c_k . a^b(x - c_k)  (+ mirror-wall terms),
// with b the component of population i.  Parameter sensitivities
// dL/dG^{ab} and dL/dtau_a are accumulated per block in FP64.
//
// Kernels: k_adj_seed (lambda^N from dL/drho at the last step),
// k_adj_local (mu gather + local reverse pass), k_adj_finish (stencil
// transpose), k_adj_rho0 (dL/drho_0 = sum_i w_i lambda^0_i for an initial
// state f^eq(rho_0, u = 0)).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kThreadsA = 256;
constexpr int kAdjBlocks = 1216;

struct Nb {
    long long cell;
    long long xo[3], yo[3], zo[3];
    bool zlo, zhi;   // z - 1 (resp. z + 1) is a wall site
};

template <class R>
__device__ __forceinline__ void nb_of(const Phys<R> &p, long long cell, Nb &n)
{
    const long long plane = (long long)p.nx * p.ny;
    const int z = (int)(cell / plane);
    const long long rem = cell - (long long)z * plane;
    const int y = (int)(rem / p.nx);
    const int x = (int)(rem - (long long)y * p.nx);
    n.cell = cell;
    n.xo[0] = x == 0 ? p.nx - 1 : x - 1;
    n.xo[1] = x;
    n.xo[2] = x == p.nx - 1 ? 0 : x + 1;
    n.yo[0] = (long long)(y == 0 ? p.ny - 1 : y - 1) * p.nx;
    n.yo[1] = (long long)y * p.nx;
    n.yo[2] = (long long)(y == p.ny - 1 ? 0 : y + 1) * p.nx;
    n.zo[0] = (long long)(z == 0 ? p.nz - 1 : z - 1) * plane;
    n.zo[1] = (long long)z * plane;
    n.zo[2] = (long long)(z == p.nz - 1 ? 0 : z + 1) * plane;
    n.zlo = p.wall_z && z == 0;
    n.zhi = p.wall_z && z == p.nz - 1;
}

__device__ __forceinline__ long long at(const Nb &n, int dx, int dy, int dz)
{
    return n.zo[1 + dz] + n.yo[1 + dy] + n.xo[1 + dx];
}

template <class R>
__device__ __forceinline__ R gradP_alpha(R cv, R vsq) { return R(3) + R(9) * cv + R(13.5) * cv * cv - R(4.5) * vsq; }
template <class R>
__device__ __forceinline__ R P_of(R cv, R vsq) { return R(1) + R(3) * cv + R(4.5) * cv * cv - R(1.5) * vsq + R(4.5) * cv * cv * cv - R(4.5) * cv * vsq; }

// One cell of the local reverse pass.
template <int S, bool REG>
__device__ void adj_cell(const typename Store<S>::T *__restrict__ f, const typename Store<S>::R *__restrict__ rho,
                         const typename Store<S>::R *__restrict__ lam_next, typename Store<S>::R *__restrict__ lam_loc,
                         typename Store<S>::R *__restrict__ aout, const Phys<typename Store<S>::R> &p, const Nb &n,
                         double (&par)[4])
{
    using R = typename Store<S>::R;
    const long long N = p.N;
    // ---- forward recomputation ------------------------------------------
    R fa[2][Q];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = (cz(i) == 1 && n.zlo) || (cz(i) == -1 && n.zhi);
            const long long idx = wall ? (long long)(a * Q + opp(i)) * N + n.cell
                                       : (long long)(a * Q + i) * N + at(n, -cx(i), -cy(i), -cz(i));
            fa[a][i] = Store<S>::load(f + idx, w<R>(i) * p.rho0);
        }
    R r[2], jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        R s = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            s += fa[a][i];
            if (cx(i) == 1) jx += fa[a][i]; else if (cx(i) == -1) jx -= fa[a][i];
            if (cy(i) == 1) jy += fa[a][i]; else if (cy(i) == -1) jy -= fa[a][i];
            if (cz(i) == 1) jz += fa[a][i]; else if (cz(i) == -1) jz -= fa[a][i];
        }
        r[a] = s;
    }
    const R rt = r[0] + r[1];
    const R u[3] = {jx / rt, jy / rt, jz / rt};
    R Sb[2][3];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        R s3[3] = {0, 0, 0};
        const R *rb = rho + (long long)b * N;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && n.zlo) || (cz(i) == 1 && n.zhi);
            R rv;
            if (wall) {
                rv = p.rho_s[b];
                if (p.wall_mirror) rv += rb[at(n, cx(i), cy(i), 0)];
            } else {
                rv = rb[at(n, cx(i), cy(i), cz(i))];
            }
            const R wr = w<R>(i) * rv;
            s3[0] += cx(i) * wr; s3[1] += cy(i) * wr; s3[2] += cz(i) * wr;
        }
        Sb[b][0] = s3[0]; Sb[b][1] = s3[1]; Sb[b][2] = s3[2];
    }
    const R Gab[2] = {p.G12, p.G21};
    R v[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) v[a][d] = u[d] + Gab[a] * Sb[1 - a][d] + p.gext[d];
    const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    // ---- mu = lambda^{n+1} gathered along +c_i -----------------------------
    R mu[2][Q];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool wall = (cz(i) == -1 && n.zlo) || (cz(i) == 1 && n.zhi);
            const long long idx = wall ? (long long)(a * Q + opp(i)) * N + n.cell
                                       : (long long)(a * Q + i) * N + at(n, cx(i), cy(i), cz(i));
            mu[a][i] = lam_next[idx];
        }

    // ---- reverse pass -------------------------------------------------------
    R lam[2][Q];
    R ubar[3] = {0, 0, 0};
    R rbar[2] = {0, 0};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const R omega = p.omega[a];
        const R keep = R(1) - omega;
        const R ra = r[a];
        const R rq = ra / R(36);
        const R vsq = v[a][0] * v[a][0] + v[a][1] * v[a][1] + v[a][2] * v[a][2];
        R Kbar = 0;            // dL/dkeep
        R vb_c[3] = {0, 0, 0}; // sum_i mu_i k_i alpha_i(v) c_i
        R vb_v = 0;            // sum_i mu_i k_i beta_i(v)
        R ub_c[3] = {0, 0, 0}; // same at u (BGK only)
        R ub_v = 0;
        R rb = 0;
        // regularized: Pi and its adjoint
        R Pi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        R tr = 0;
        if (REG) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int c[3] = {cx(i), cy(i), cz(i)};
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) Pi[x][y] += R(c[x] * c[y]) * fa[a][i];
            }
            const R T0 = R(1) / R(3);
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) Pi[x][y] -= ra * ((x == y ? T0 : R(0)) + u[x] * u[y]);
            tr = Pi[0][0] + Pi[1][1] + Pi[2][2];
        }
        R Pbar[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int c[3] = {cx(i), cy(i), cz(i)};
            const R ki = R(k36(i));
            const R m = mu[a][i];
            const R cv = R(c[0]) * v[a][0] + R(c[1]) * v[a][1] + R(c[2]) * v[a][2];
            // E_i(rho, v) = rq k_i P_i(v)
            rb += m * (ki / R(36)) * P_of(cv, vsq);
            const R mk = m * ki;
            const R al = gradP_alpha(cv, vsq), be = R(3) + R(9) * cv;
#pragma unroll
            for (int d = 0; d < 3; ++d) vb_c[d] += mk * al * R(c[d]);
            vb_v += mk * be;
            if (!REG) {
                const R cu = R(c[0]) * u[0] + R(c[1]) * u[1] + R(c[2]) * u[2];
                const R Eu = rq * ki * P_of(cu, usq);
                // f* = E(rho, v) + keep (f - E(rho, u))
                lam[a][i] = keep * m;
                Kbar += m * (fa[a][i] - Eu);
                rb -= keep * m * (ki / R(36)) * P_of(cu, usq);
                const R alu = gradP_alpha(cu, usq), beu = R(3) + R(9) * cu;
#pragma unroll
                for (int d = 0; d < 3; ++d) ub_c[d] += mk * alu * R(c[d]);
                ub_v += mk * beu;
            } else {
                // f* = E(rho, v) + keep (k_i/8) (c c : Pi - tr Pi / 3)
                R ccP = 0;
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) ccP += R(c[x] * c[y]) * Pi[x][y];
                const R Ni = ki * R(0.125) * (ccP - tr / R(3));
                Kbar += m * Ni;
                const R nb = keep * m * ki * R(0.125);
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) Pbar[x][y] += nb * (R(c[x] * c[y]) - (x == y ? R(1) / R(3) : R(0)));
                lam[a][i] = 0;
            }
        }
        // dL/dv^a, dL/du (through E(rho, u) for BGK), dL/drho^a
        R vbar[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) vbar[d] = rq * (vb_c[d] - v[a][d] * vb_v);
        if (!REG) {
#pragma unroll
            for (int d = 0; d < 3; ++d) ubar[d] += -keep * rq * (ub_c[d] - u[d] * ub_v);
        } else {
            // Pi = sum c c f - rho (T0 I + u u)
            const R T0 = R(1) / R(3);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int c[3] = {cx(i), cy(i), cz(i)};
                R s = 0;
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) s += Pbar[x][y] * R(c[x] * c[y]);
                lam[a][i] += s;
            }
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) {
                    rb -= Pbar[x][y] * ((x == y ? T0 : R(0)) + u[x] * u[y]);
                    ubar[x] -= ra * Pbar[x][y] * u[y];
                    ubar[y] -= ra * Pbar[x][y] * u[x];
                }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) ubar[d] += vbar[d];
        rbar[a] = rb;
        // g^a = G^{ab} S^b + g_ext:  dL/dS^b = G^{ab} vbar,  dL/dG^{ab} = vbar . S^b
        const int b = 1 - a;
#pragma unroll
        for (int d = 0; d < 3; ++d) aout[((long long)b * 3 + d) * N + n.cell] = Gab[a] * vbar[d];
        par[a] += (double)(vbar[0] * Sb[b][0] + vbar[1] * Sb[b][1] + vbar[2] * Sb[b][2]);
        // keep = 1 - 1/tau: dkeep/dtau = 1/tau^2
        par[2 + a] += (double)(Kbar * omega * omega);
    }
    // u = j / rho: dL/dj = ubar / rho, dL/drho += -(ubar . u) / rho
    const R jb[3] = {ubar[0] / rt, ubar[1] / rt, ubar[2] / rt};
    const R rtb = -(ubar[0] * u[0] + ubar[1] * u[1] + ubar[2] * u[2]) / rt;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i)
            lam_loc[(long long)(a * Q + i) * N + n.cell] =
                lam[a][i] + rbar[a] + rtb + R(cx(i)) * jb[0] + R(cy(i)) * jb[1] + R(cz(i)) * jb[2];
}

template <int S, bool REG>
__global__ void __launch_bounds__(kThreadsA)
k_adj_local(const typename Store<S>::T *__restrict__ f, const typename Store<S>::R *__restrict__ rho,
            const typename Store<S>::R *__restrict__ lam_next, typename Store<S>::R *__restrict__ lam_loc,
            typename Store<S>::R *__restrict__ aout, double *__restrict__ partials, Phys<typename Store<S>::R> p)
{
    double par[4] = {0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * kThreadsA + threadIdx.x; c < p.N;
         c += (long long)gridDim.x * kThreadsA) {
        Nb n;
        nb_of(p, c, n);
        adj_cell<S, REG>(f, rho, lam_next, lam_loc, aout, p, n, par);
    }
    __shared__ double sh[4][kThreadsA];
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = par[k];
    __syncthreads();
    for (int s = kThreadsA / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[(long long)blockIdx.x * 4 + threadIdx.x] += sh[threadIdx.x][0];
}

// lambda^n = lambda_loc + D^b(x), D^b(x) = sum_k w_k c_k . a^b(x - c_k), plus
// the mirror-wall terms: a wall site x' + c_k seen from x' presents the
// density of its mirror cell x' + (c_kx, c_ky, 0).
template <class R>
__global__ void __launch_bounds__(kThreadsA)
k_adj_finish(const R *__restrict__ lam_loc, const R *__restrict__ a, R *__restrict__ lam, Phys<R> p)
{
    const long long c = (long long)blockIdx.x * kThreadsA + threadIdx.x;
    if (c >= p.N) return;
    Nb n;
    nb_of(p, c, n);
    const long long N = p.N;
    R D[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        R s = 0;
        const R *ab = a + (long long)b * 3 * N;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            // regular term: x - c_k is a fluid cell whose neighbour x + 0 is this cell
            const bool src_wall = (cz(k) == 1 && n.zlo) || (cz(k) == -1 && n.zhi);
            if (!src_wall) {
                const long long src = at(n, -cx(k), -cy(k), -cz(k));
                s += w<R>(k) * (R(cx(k)) * ab[src] + R(cy(k)) * ab[N + src] + R(cz(k)) * ab[2 * N + src]);
            }
            // mirror term: the cell y = x - (c_kx, c_ky, 0) of this plane sees the
            // wall site y + c_k, whose density is this cell's
            if (p.wall_mirror) {
                const bool mirror = (cz(k) == -1 && n.zlo) || (cz(k) == 1 && n.zhi);
                if (mirror) {
                    const long long src = at(n, -cx(k), -cy(k), 0);
                    s += w<R>(k) * (R(cx(k)) * ab[src] + R(cy(k)) * ab[N + src] + R(cz(k)) * ab[2 * N + src]);
                }
            }
        }
        D[b] = s;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long idx = (long long)(b * Q + i) * N + c;
            lam[idx] = lam_loc[idx] + D[b];
        }
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

template <class R>
__global__ void __launch_bounds__(kThreadsA)
k_adj_rho0(const R *__restrict__ lam, double *__restrict__ g1, double *__restrict__ g2, long long N)
{
    const long long c = (long long)blockIdx.x * kThreadsA + threadIdx.x;
    if (c >= N) return;
    double s1 = 0, s2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s1 += wd(i) * (double)lam[(long long)i * N + c];
        s2 += wd(i) * (double)lam[(long long)(Q + i) * N + c];
    }
    if (g1) g1[c] = s1;
    if (g2) g2[c] = s2;
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
    return p;
}

inline unsigned gridA(long long N) { return (unsigned)((N + kThreadsA - 1) / kThreadsA); }

template <int S>
cudaError_t adj_step_t(const HostPhys &h, const void *f, const void *rho, const void *lam_next, void *lam_loc,
                       void *a, void *lam_out, double *partials, cudaStream_t s)
{
    using T = typename Store<S>::T;
    using R = typename Store<S>::R;
    const Phys<R> p = make_phys_a<R>(h);
    if (h.collision == LBM_REGULARIZED)
        k_adj_local<S, true><<<kAdjBlocks, kThreadsA, 0, s>>>((const T *)f, (const R *)rho, (const R *)lam_next,
                                                              (R *)lam_loc, (R *)a, partials, p);
    else
        k_adj_local<S, false><<<kAdjBlocks, kThreadsA, 0, s>>>((const T *)f, (const R *)rho, (const R *)lam_next,
                                                               (R *)lam_loc, (R *)a, partials, p);
    k_adj_finish<R><<<gridA(h.N), kThreadsA, 0, s>>>((const R *)lam_loc, (const R *)a, (R *)lam_out, p);
    return cudaGetLastError();
}

}  // namespace

int adjoint_blocks() { return kAdjBlocks; }

cudaError_t launch_adjoint_step(const HostPhys &p, const void *f, const void *rho, const void *lam_next,
                                void *lam_loc, void *a, void *lam_out, double *partials, cudaStream_t s)
{
    switch (p.storage) {
    case ST_F64: return adj_step_t<ST_F64>(p, f, rho, lam_next, lam_loc, a, lam_out, partials, s);
    case ST_F32: return adj_step_t<ST_F32>(p, f, rho, lam_next, lam_loc, a, lam_out, partials, s);
    case ST_F16_DEV: return adj_step_t<ST_F16_DEV>(p, f, rho, lam_next, lam_loc, a, lam_out, partials, s);
    case ST_BF16_DEV: return adj_step_t<ST_BF16_DEV>(p, f, rho, lam_next, lam_loc, a, lam_out, partials, s);
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

cudaError_t launch_adjoint_rho0(const HostPhys &p, const void *lam, double *g1, double *g2, cudaStream_t s)
{
    if (p.storage == ST_F64)
        k_adj_rho0<double><<<gridA(p.N), kThreadsA, 0, s>>>((const double *)lam, g1, g2, p.N);
    else
        k_adj_rho0<float><<<gridA(p.N), kThreadsA, 0, s>>>((const float *)lam, g1, g2, p.N);
    return cudaGetLastError();
}

}  // namespace lbm
