// C ABI of the library (declared in include/lbm.h): argument validation,
// device memory, the stream, and the order of kernel launches of a time step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <utility>
#include <algorithm>
#include <vector>

#include "../../include/lbm.h"
#include "d3q19.cuh"
#include "lbm_internal.h"

struct lbm_lattice {
    lbm_params params;
    lbm::HostPhys phys;
    int device;
    cudaStream_t stream;
    bool own_stream;
    void *f[2];          // population copies (storage format)
    int cur;             // index of the copy holding the current state
    void *rho;           // density scratch of the two-kernel step (2*N reals)
    double *partials;    // reduction partials (device)
    double *partials_h;  // reduction partials (pinned host)
    long steps;
    int use_fused;
    int init_at_rest;    // current run started from lbm_init_fields with u = NULL
    // recording for the reverse pass
    void *ckpt;          // checkpoint store (rec_nck raw states)
    long rec_steps;
    int rec_every;
    long rec_nck;
    int rec_at_rest;     // the recording started at rest right after lbm_init_fields
    // working memory of the reverse pass, reserved by lbm_record: lambda_loc
    // (two, ping-pong), a, D (two), one segment of states and of their
    // densities, gradient staging, partials
    void *ws_lam, *ws_lam_loc, *ws_a, *ws_d, *ws_seg, *ws_rseg, *ws_io;
    double *ws_part;
    // CUDA graphs of one full checkpoint segment of the reverse pass, one per
    // ping-pong parity of the adjoint fields (0 not built, -1 not available)
    cudaGraphExec_t seg_graph[2];
    int seg_graph_state[2];
    // CUDA graph of kGraphSteps steps from copy 0 (replayed by lbm_step)
    cudaGraphExec_t graph;
    int graph_state;     // 0 not built, 1 ready, -1 not available (plain launches)
    int use_graphs;
    unsigned char *solid;   // device mask of solid sites (N bytes) or nullptr
    unsigned *links;        // its link flags (N words) or nullptr
    // fused step under the mask: wall densities (N pairs) and the boundary
    // cells of the mirror model (see HostPhys)
    float *wall_rho;
    unsigned *bfluid, *bsolid;
};

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
lbm_status fail(lbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

lbm_status cuda_fail(cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(LBM_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr, where)                                   \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// Make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

bool env_flag(const char *name, int dflt)
{
    const char *v = getenv(name);
    if (!v || !*v) return dflt != 0;
    return atoi(v) != 0;
}

lbm_status copy_in(const lbm_lattice *h, void *dst, const void *src, size_t bytes, int on_device)
{
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream),
       "copy to device");
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_lattice_dirs(int c[19][3], double w[19])
{
    for (int i = 0; i < lbm::Q; ++i) {
        if (c) {
            c[i][0] = lbm::cx(i);
            c[i][1] = lbm::cy(i);
            c[i][2] = lbm::cz(i);
        }
        if (w) w[i] = lbm::wd(i);
    }
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params *pp, lbm_lattice **out)
{
    if (!pp || !out) return fail(LBM_EINVAL, "lbm_create: NULL argument");
    *out = nullptr;
    const lbm_params &p = *pp;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1)
        return fail(LBM_EINVAL, "lbm_create: sizes must be >= 1 (got %d x %d x %d)", p.nx, p.ny, p.nz);
    const long long N = (long long)p.nx * p.ny * p.nz;
    if (N > (1LL << 40)) return fail(LBM_EINVAL, "lbm_create: lattice too large");
    for (int a = 0; a < 2; ++a)
        if (!(p.tau[a] > 0.5) || !isfinite(p.tau[a]))
            return fail(LBM_EINVAL, "lbm_create: tau[%d] = %g must be a finite value > 1/2", a, p.tau[a]);
    if (p.G[0][0] != 0.0 || p.G[1][1] != 0.0)
        return fail(LBM_ENOTSUP, "lbm_create: G^{aa} must be 0 (single-component phase transitions are "
                                 "excluded)");
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (!isfinite(p.G[a][b])) return fail(LBM_EINVAL, "lbm_create: G must be finite");
    for (int d = 0; d < 3; ++d)
        if (!isfinite(p.g_ext[d])) return fail(LBM_EINVAL, "lbm_create: g_ext must be finite");
    if (!isfinite(p.rho_s[0]) || !isfinite(p.rho_s[1]) || !isfinite(p.rho0_dev))
        return fail(LBM_EINVAL, "lbm_create: rho_s and rho0_dev must be finite");
    if (p.storage < LBM_F64 || p.storage > LBM_BF16_REL)
        return fail(LBM_EINVAL, "lbm_create: unknown storage %d", p.storage);
    if (p.storage != LBM_F16_DEV && p.storage != LBM_BF16_DEV && p.rho0_dev != 0.0)
        return fail(LBM_EINVAL, "lbm_create: rho0_dev applies to the 16-bit deviation formats only");
    if (p.collision != LBM_BGK && p.collision != LBM_REGULARIZED && p.collision != LBM_REGULARIZED3)
        return fail(LBM_EINVAL, "lbm_create: unknown collision %d", p.collision);
    if (p.wall_model != LBM_WALL_POTENTIAL && p.wall_model != LBM_WALL_MIRROR)
        return fail(LBM_EINVAL, "lbm_create: unknown wall model %d", p.wall_model);
    if (p.forcing != LBM_FORCING_EDM && p.forcing != LBM_FORCING_GUO)
        return fail(LBM_EINVAL, "lbm_create: unknown forcing %d", p.forcing);
    for (int d = 0; d < 3; ++d)
        if (p.periodic[d] != 0 && p.periodic[d] != 1)
            return fail(LBM_EINVAL, "lbm_create: periodic[%d] must be 0 or 1", d);
    if (!p.periodic[0] || !p.periodic[1])
        return fail(LBM_ENOTSUP, "lbm_create: walls are supported along z only");

    lbm_lattice *h = (lbm_lattice *)calloc(1, sizeof(lbm_lattice));
    if (!h) return fail(LBM_ENOMEM, "lbm_create: host allocation failed");
    h->params = p;
    lbm::HostPhys &ph = h->phys;
    ph.nx = p.nx; ph.ny = p.ny; ph.nz = p.nz; ph.N = N;
    ph.wall_z = p.periodic[2] ? 0 : 1;
    ph.wall_mirror = p.wall_model == LBM_WALL_MIRROR;
    ph.storage = p.storage;
    ph.collision = p.collision;
    ph.forcing = p.forcing;
    ph.tau[0] = p.tau[0]; ph.tau[1] = p.tau[1];
    ph.G12 = p.G[0][1]; ph.G21 = p.G[1][0];
    for (int d = 0; d < 3; ++d) ph.gext[d] = p.g_ext[d];
    ph.rho_s[0] = p.rho_s[0]; ph.rho_s[1] = p.rho_s[1];
    ph.rho0 = p.rho0_dev;
    ph.ref_off = (long long)lbm::ref_offset(p.storage, N);
    h->use_fused = env_flag("LBM_FUSED", 1) && lbm::fused_supported(ph);
    h->use_graphs = env_flag("LBM_GRAPHS", 1);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { free(h); return cuda_fail(e, "lbm_create: cudaGetDevice"); }
    if (p.stream) {
        h->stream = (cudaStream_t)p.stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { free(h); return cuda_fail(e, "lbm_create: stream"); }
        h->own_stream = true;
    }
    const size_t pop_bytes = lbm::state_bytes(p.storage, N);   // populations (+ references)
    const size_t rho_bytes = (size_t)2 * (size_t)N * lbm::real_bytes(p.storage);
    const int nb = lbm::reduce_blocks();
    if ((e = cudaMalloc(&h->f[0], pop_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->f[1], pop_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&h->rho, rho_bytes)) != cudaSuccess ||
        (e = cudaMalloc((void **)&h->partials, (size_t)nb * 8 * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost((void **)&h->partials_h, (size_t)nb * 8 * sizeof(double))) != cudaSuccess) {
        lbm_status st = cuda_fail(e, "lbm_create: allocation");
        lbm_destroy(h);
        return st;
    }
    // A fresh lattice holds the uniform state rho^1 = rho^2 = 0 until initialised:
    // zero the populations so that nothing reads uninitialised memory.
    if ((e = cudaMemsetAsync(h->f[0], 0, pop_bytes, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->f[1], 0, pop_bytes, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
        lbm_status st = cuda_fail(e, "lbm_create: clear");
        lbm_destroy(h);
        return st;
    }
    h->cur = 0;
    h->steps = 0;
    *out = h;
    return LBM_OK;
}

namespace {

void free_workspace(lbm_lattice *h)
{
    void *bufs[8] = {h->ws_lam, h->ws_lam_loc, h->ws_a, h->ws_d, h->ws_seg, h->ws_rseg, h->ws_io, h->ws_part};
    for (void *b : bufs) cudaFree(b);
    for (int q = 0; q < 2; ++q) {
        if (h->seg_graph[q]) cudaGraphExecDestroy(h->seg_graph[q]);
        h->seg_graph[q] = nullptr;
        h->seg_graph_state[q] = 0;
    }
    h->ws_lam = h->ws_lam_loc = h->ws_a = h->ws_d = h->ws_seg = h->ws_rseg = h->ws_io = nullptr;
    h->ws_part = nullptr;
}

}  // namespace

namespace {

// Releases a lattice's mask and everything derived from it.
void free_mask(lbm_lattice *h)
{
    void *bufs[5] = {h->solid, h->links, h->wall_rho, h->bfluid, h->bsolid};
    for (void *b : bufs) cudaFree(b);
    h->solid = nullptr;
    h->links = nullptr;
    h->wall_rho = nullptr;
    h->bfluid = h->bsolid = nullptr;
    h->phys.solid = nullptr;
    h->phys.links = nullptr;
    h->phys.wall_rho = nullptr;
    h->phys.bfluid = h->phys.bsolid = nullptr;
    h->phys.n_bfluid = h->phys.n_bsolid = 0;
}

}  // namespace

void lbm_destroy(lbm_lattice *h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->f[0]);
    cudaFree(h->f[1]);
    cudaFree(h->rho);
    cudaFree(h->ckpt);
    free_workspace(h);
    free_mask(h);
    cudaFree(h->partials);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->partials_h) cudaFreeHost(h->partials_h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    free(h);
}

lbm_status lbm_init_fields(lbm_lattice *h, const double *rho1, const double *rho2, const double *u,
                           int on_device)
{
    if (!h || !rho1 || !rho2) return fail(LBM_EINVAL, "lbm_init_fields: NULL argument");
    DeviceGuard g(h->device);
    const size_t N = (size_t)h->phys.N;
    const double *d1 = rho1, *d2 = rho2, *du = u;
    // The other state copy is free until the first step: it stages host fields
    // (no allocation) and then holds the rest values of a state at rest.
    char *spare = (char *)h->f[1];
    const size_t cap = lbm::state_bytes(h->phys.storage, N);
    const size_t stage = on_device ? 0 : sizeof(double) * N * (u ? 5 : 2);
    const size_t rest = 8 * N * lbm::real_bytes(h->phys.storage);
    void *tmp = nullptr;
    if (!on_device) {
        double *t = (double *)spare;
        if (stage + rest > cap) {   // not reached by the built formats (at most 104 of 304 B per cell)
            CK(cudaMallocAsync(&tmp, stage, h->stream), "lbm_init_fields: staging");
            t = (double *)tmp;
        }
        lbm_status st;
        if ((st = copy_in(h, t, rho1, sizeof(double) * N, 0)) != LBM_OK) return st;
        if ((st = copy_in(h, t + N, rho2, sizeof(double) * N, 0)) != LBM_OK) return st;
        if (u && (st = copy_in(h, t + 2 * N, u, sizeof(double) * 3 * N, 0)) != LBM_OK) return st;
        d1 = t;
        d2 = t + N;
        du = u ? t + 2 * N : nullptr;
    }
    h->cur = 0;
    h->steps = 0;
    h->init_at_rest = u == nullptr;
    void *scratch = tmp ? (void *)spare : (stage + rest <= cap ? (void *)(spare + stage) : nullptr);
    CK(lbm::launch_init_feq(h->phys, d1, d2, du, h->f[0], scratch, h->stream), "lbm_init_fields: launch");
    if (tmp) CK(cudaFreeAsync(tmp, h->stream), "lbm_init_fields: free staging");
    // host inputs: the caller may reuse its buffers on return
    if (!on_device) CK(cudaStreamSynchronize(h->stream), "lbm_init_fields: sync");
    return LBM_OK;
}

namespace {

// Steps per graph launch; even, so that a replay leaves the state in copy 0.
constexpr long kGraphSteps = 16;

cudaError_t launch_one(lbm_lattice *h, int from, cudaStream_t s)
{
    return h->use_fused ? lbm::launch_step_fused(h->phys, h->f[from], h->f[from ^ 1], s)
                        : lbm::launch_step_split(h->phys, h->f[from], h->f[from ^ 1], h->rho, s);
}

// Captures kGraphSteps ping-pong steps starting from copy 0 on a private
// stream (the lattice's stream may be the legacy default stream, which cannot
// be captured) and instantiates them.  On any failure the lattice keeps
// plain launches.
bool build_graph(lbm_lattice *h)
{
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t gr = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        for (long t = 0; t < kGraphSteps && ok; ++t) ok = launch_one(h, (int)(t & 1), cs) == cudaSuccess;
        const cudaError_t e = cudaStreamEndCapture(cs, &gr);
        ok = ok && e == cudaSuccess && gr != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(&h->graph, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!ok) h->graph = nullptr;
    return ok;
}

}  // namespace

lbm_status lbm_step(lbm_lattice *h, long n_steps)
{
    if (!h) return fail(LBM_EINVAL, "lbm_step: NULL handle");
    if (n_steps < 0) return fail(LBM_EINVAL, "lbm_step: n_steps = %ld < 0", n_steps);
    DeviceGuard g(h->device);
    long t = 0;
    auto plain = [&](long upto) -> lbm_status {
        for (; t < upto; ++t) {
            const cudaError_t e = launch_one(h, h->cur, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "lbm_step: launch");
            h->cur ^= 1;
            ++h->steps;
        }
        return LBM_OK;
    };
    // long runs replay a captured graph of kGraphSteps steps (one launch per
    // graph instead of one or two per step); the first steps run plainly, so
    // that every kernel has been launched once before the capture
    if (h->use_graphs && h->graph_state >= 0 && n_steps >= 2 * kGraphSteps + 2) {
        lbm_status st = plain(h->cur == 1 ? 1 : 2);
        if (st != LBM_OK) return st;
        if (h->graph_state == 0) h->graph_state = build_graph(h) ? 1 : -1;
        if (h->graph_state == 1) {
            for (; n_steps - t >= kGraphSteps; t += kGraphSteps) {
                const cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "lbm_step: graph launch");
                h->steps += kGraphSteps;
            }
        }
    }
    return plain(n_steps);
}

lbm_status lbm_step_timed(lbm_lattice *h, long n_steps, double kernel_ms[4], long launches[4],
                          const char *names[4], int *n_kinds)
{
    if (!h || !kernel_ms || !launches || !names || !n_kinds)
        return fail(LBM_EINVAL, "lbm_step_timed: NULL argument");
    if (n_steps <= 0) return fail(LBM_EINVAL, "lbm_step_timed: n_steps = %ld must be > 0", n_steps);
    DeviceGuard g(h->device);
    const int kinds = h->use_fused ? 1 : 2;
    const size_t nev = (size_t)n_steps * (kinds + 1);
    std::vector<cudaEvent_t> ev(nev, nullptr);
    lbm_status st = LBM_OK;
    for (size_t k = 0; k < nev && st == LBM_OK; ++k) {
        cudaError_t e = cudaEventCreate(&ev[k]);
        if (e != cudaSuccess) st = cuda_fail(e, "lbm_step_timed: event");
    }
    for (long t = 0; t < n_steps && st == LBM_OK; ++t) {
        cudaEvent_t *evt = &ev[(size_t)t * (kinds + 1)];
        cudaError_t e;
        if (h->use_fused)
            e = lbm::launch_step_fused(h->phys, h->f[h->cur], h->f[h->cur ^ 1], h->stream, evt);
        else
            e = lbm::launch_step_split(h->phys, h->f[h->cur], h->f[h->cur ^ 1], h->rho, h->stream, evt);
        if (e != cudaSuccess) { st = cuda_fail(e, "lbm_step_timed: launch"); break; }
        h->cur ^= 1;
        ++h->steps;
    }
    if (st == LBM_OK) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "lbm_step_timed: sync");
    }
    if (st == LBM_OK) {
        static const char *kFused[1] = {"k_step_fused"};
        static const char *kSplit[2] = {"k_density", "k_collide"};
        for (int k = 0; k < 4; ++k) { kernel_ms[k] = 0; launches[k] = 0; names[k] = nullptr; }
        for (long t = 0; t < n_steps && st == LBM_OK; ++t)
            for (int k = 0; k < kinds; ++k) {
                float ms = 0;
                cudaError_t e = cudaEventElapsedTime(&ms, ev[(size_t)t * (kinds + 1) + k],
                                                     ev[(size_t)t * (kinds + 1) + k + 1]);
                if (e != cudaSuccess) { st = cuda_fail(e, "lbm_step_timed: elapsed"); break; }
                kernel_ms[k] += ms;
                launches[k] += 1;
            }
        for (int k = 0; k < kinds; ++k) names[k] = h->use_fused ? kFused[k] : kSplit[k];
        *n_kinds = kinds;
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    return st;
}

lbm_status lbm_moments(lbm_lattice *h, int out_f64, void *rho1, void *rho2, void *uF, int on_device)
{
    if (!h) return fail(LBM_EINVAL, "lbm_moments: NULL handle");
    if (!rho1 && !rho2 && !uF) return LBM_OK;
    DeviceGuard g(h->device);
    const size_t N = (size_t)h->phys.N;
    const size_t es = out_f64 ? 8 : 4;
    if (on_device) {
        CK(lbm::launch_moments(h->phys, h->f[h->cur], h->rho, out_f64, rho1, rho2, uF, h->stream),
           "lbm_moments: launch");
        return LBM_OK;
    }
    void *tmp = nullptr;
    CK(cudaMallocAsync(&tmp, es * N * 5, h->stream), "lbm_moments: staging");
    char *t = (char *)tmp;
    CK(lbm::launch_moments(h->phys, h->f[h->cur], h->rho, out_f64, rho1 ? t : nullptr,
                           rho2 ? t + es * N : nullptr, uF ? t + 2 * es * N : nullptr, h->stream),
       "lbm_moments: launch");
    if (rho1) CK(cudaMemcpyAsync(rho1, t, es * N, cudaMemcpyDeviceToHost, h->stream), "lbm_moments: copy");
    if (rho2) CK(cudaMemcpyAsync(rho2, t + es * N, es * N, cudaMemcpyDeviceToHost, h->stream), "lbm_moments: copy");
    if (uF) CK(cudaMemcpyAsync(uF, t + 2 * es * N, 3 * es * N, cudaMemcpyDeviceToHost, h->stream), "lbm_moments: copy");
    CK(cudaFreeAsync(tmp, h->stream), "lbm_moments: free staging");
    CK(cudaStreamSynchronize(h->stream), "lbm_moments: sync");
    return LBM_OK;
}

lbm_status lbm_reduce(lbm_lattice *h, double out[6])
{
    if (!h || !out) return fail(LBM_EINVAL, "lbm_reduce: NULL argument");
    DeviceGuard g(h->device);
    const int nb = lbm::reduce_blocks();
    CK(lbm::launch_reduce(h->phys, h->f[h->cur], h->rho, h->partials, h->stream), "lbm_reduce: launch");
    CK(cudaMemcpyAsync(h->partials_h, h->partials, (size_t)nb * 8 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream),
       "lbm_reduce: copy");
    CK(cudaStreamSynchronize(h->stream), "lbm_reduce: sync");
    double acc[6] = {0, 0, 0, 0, 0, 0}, bad = 0;
    for (int b = 0; b < nb; ++b) {
        const double *q = h->partials_h + (size_t)b * 8;
        for (int k = 0; k < 5; ++k) acc[k] += q[k];
        acc[5] = fmax(acc[5], q[5]);
        bad += q[6];
    }
    for (int k = 0; k < 5; ++k) out[k] = acc[k];
    out[5] = sqrt(acc[5]);   // the blocks reduce max |u_F|^2
    if (bad > 0 || !isfinite(acc[0]) || !isfinite(acc[1]))
        return fail(LBM_ENUMERIC, "lbm_reduce: %.0f cells with a non-finite or non-positive density", bad);
    return LBM_OK;
}

namespace {

lbm_status diag_run(lbm_lattice *h, int which, const double *vec3, double a0, double a1, double *sums, int nsums)
{
    const int nb = lbm::diag_blocks(), ns = lbm::diag_slots();
    CK(lbm::launch_density(h->phys, h->f[h->cur], h->rho, h->stream), "diagnostics: density");
    if (which == 0)
        CK(lbm::launch_pressure(h->phys, h->rho, vec3, a0, a1, h->partials, h->stream), "diagnostics: pressure");
    else
        CK(lbm::launch_droplet(h->phys, h->rho, a0, vec3, h->partials, h->stream), "diagnostics: droplet");
    CK(cudaMemcpyAsync(h->partials_h, h->partials, sizeof(double) * (size_t)nb * ns, cudaMemcpyDeviceToHost,
                       h->stream),
       "diagnostics: copy");
    CK(cudaStreamSynchronize(h->stream), "diagnostics: sync");
    for (int k = 0; k < nsums; ++k) sums[k] = 0;
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < nsums; ++k) sums[k] += h->partials_h[(size_t)b * ns + k];
    return LBM_OK;
}

}  // namespace

lbm_status lbm_pressure_jump(lbm_lattice *h, const double center[3], double r_in, double r_out, double out[3])
{
    if (!h || !center || !out) return fail(LBM_EINVAL, "lbm_pressure_jump: NULL argument");
    if (!(r_in > 0) || !(r_out >= r_in)) return fail(LBM_EINVAL, "lbm_pressure_jump: need 0 < r_in <= r_out");
    DeviceGuard g(h->device);
    double s[4] = {0, 0, 0, 0};
    lbm_status st = diag_run(h, 0, center, r_in, r_out, s, 4);
    if (st != LBM_OK) return st;
    if (s[1] < 1 || s[3] < 1) return fail(LBM_EINVAL, "lbm_pressure_jump: empty inner or outer region");
    out[0] = s[0] / s[1];
    out[1] = s[2] / s[3];
    out[2] = out[0] - out[1];
    return LBM_OK;
}

lbm_status lbm_droplet_stats(lbm_lattice *h, double threshold, const double origin[3], double out[7])
{
    if (!h || !origin || !out) return fail(LBM_EINVAL, "lbm_droplet_stats: NULL argument");
    DeviceGuard g(h->device);
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    lbm_status st = diag_run(h, 1, origin, threshold, 0.0, s, 7);
    if (st != LBM_OK) return st;
    out[0] = s[0];
    for (int d = 0; d < 3; ++d) out[1 + d] = s[0] > 0 ? s[1 + d] / s[0] : 0.0;
    out[4] = s[4];
    out[5] = s[6] > 0 ? s[5] / s[6] : 0.0;
    out[6] = s[6];
    return LBM_OK;
}

lbm_status lbm_set_solid(lbm_lattice *h, const unsigned char *solid, int on_device)
{
    if (!h) return fail(LBM_EINVAL, "lbm_set_solid: NULL handle");
    if (solid && h->phys.wall_z)
        return fail(LBM_ENOTSUP, "lbm_set_solid: a mask needs a lattice periodic along z (walls are given "
                                 "either as z walls or as a mask)");
    DeviceGuard g(h->device);
    CK(cudaStreamSynchronize(h->stream), "lbm_set_solid: sync");
    // the captured step graph and any recording belong to the old geometry
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_state = 0;
    cudaFree(h->ckpt);
    h->ckpt = nullptr;
    h->rec_steps = 0;
    free_workspace(h);
    free_mask(h);
    if (!solid) {
        h->use_fused = env_flag("LBM_FUSED", 1) && lbm::fused_supported(h->phys);
        return LBM_OK;
    }
    const size_t N = (size_t)h->phys.N;
    CK(cudaMalloc((void **)&h->solid, N), "lbm_set_solid: mask");
    CK(cudaMalloc((void **)&h->links, N * sizeof(unsigned)), "lbm_set_solid: link flags");
    CK(cudaMemcpyAsync(h->solid, solid, N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream), "lbm_set_solid: copy");
    CK(lbm::launch_link_flags(h->phys, h->solid, h->links, h->stream), "lbm_set_solid: link flags");
    h->phys.solid = h->solid;
    h->phys.links = h->links;
    h->use_fused = env_flag("LBM_FUSED", 1) && lbm::fused_supported(h->phys);
    {
        // wall densities (fused step) and the boundary lists of the mirror
        // model (fused step and reverse pass): count, then list
        unsigned long long *cnt = nullptr, cnt_h[2] = {0, 0};
        CK(cudaMalloc((void **)&h->wall_rho, 2 * N * sizeof(float)), "lbm_set_solid: wall densities");
        CK(cudaMemsetAsync(h->wall_rho, 0, 2 * N * sizeof(float), h->stream), "lbm_set_solid: wall densities");
        CK(cudaMalloc((void **)&cnt, 2 * sizeof(unsigned long long)), "lbm_set_solid: counters");
        cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess)
            e = lbm::launch_mask_setup(h->phys, h->solid, h->wall_rho, nullptr, nullptr, cnt, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cnt_h, cnt, sizeof cnt_h, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->bfluid, sizeof(unsigned) * (cnt_h[0] ? cnt_h[0] : 1));
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->bsolid, sizeof(unsigned) * (cnt_h[1] ? cnt_h[1] : 1));
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess)
            e = lbm::launch_mask_setup(h->phys, h->solid, h->wall_rho, h->bfluid, h->bsolid, cnt, h->stream);
        // the lists come out in the order of the counters' atomics: sorted by
        // cell, the wall-density kernels gather along rows
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            unsigned *lst = q == 0 ? h->bfluid : h->bsolid;
            std::vector<unsigned> v((size_t)cnt_h[q]);
            if (v.empty()) continue;
            e = cudaMemcpyAsync(v.data(), lst, v.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) break;
            std::sort(v.begin(), v.end());
            e = cudaMemcpyAsync(lst, v.data(), v.size() * sizeof(unsigned), cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(cnt);
        if (e != cudaSuccess) {
            free_mask(h);
            return cuda_fail(e, "lbm_set_solid: boundary lists");
        }
        h->phys.wall_rho = h->wall_rho;
        h->phys.bfluid = h->bfluid;
        h->phys.bsolid = h->bsolid;
        h->phys.n_bfluid = (long long)cnt_h[0];
        h->phys.n_bsolid = (long long)cnt_h[1];
    }
    CK(cudaStreamSynchronize(h->stream), "lbm_set_solid: sync");
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_lattice *h, double *out, int on_device)
{
    if (!h || !out) return fail(LBM_EINVAL, "lbm_get_populations: NULL argument");
    DeviceGuard g(h->device);
    const size_t bytes = sizeof(double) * 2 * lbm::Q * (size_t)h->phys.N;
    if (on_device) {
        CK(lbm::launch_get_populations(h->phys, h->f[h->cur], out, h->stream), "lbm_get_populations");
        return LBM_OK;
    }
    void *tmp = nullptr;
    CK(cudaMallocAsync(&tmp, bytes, h->stream), "lbm_get_populations: staging");
    CK(lbm::launch_get_populations(h->phys, h->f[h->cur], (double *)tmp, h->stream), "lbm_get_populations");
    CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream), "lbm_get_populations: copy");
    CK(cudaFreeAsync(tmp, h->stream), "lbm_get_populations: free");
    CK(cudaStreamSynchronize(h->stream), "lbm_get_populations: sync");
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_lattice *h, const double *in, int on_device)
{
    if (!h || !in) return fail(LBM_EINVAL, "lbm_set_populations: NULL argument");
    DeviceGuard g(h->device);
    const size_t bytes = sizeof(double) * 2 * lbm::Q * (size_t)h->phys.N;
    const double *src = in;
    void *tmp = nullptr;
    if (!on_device) {
        CK(cudaMallocAsync(&tmp, bytes, h->stream), "lbm_set_populations: staging");
        lbm_status st = copy_in(h, tmp, in, bytes, 0);
        if (st != LBM_OK) return st;
        src = (const double *)tmp;
    }
    h->init_at_rest = 0;
    CK(lbm::launch_set_populations(h->phys, src, h->f[h->cur], h->stream), "lbm_set_populations");
    if (tmp) {
        CK(cudaFreeAsync(tmp, h->stream), "lbm_set_populations: free");
        CK(cudaStreamSynchronize(h->stream), "lbm_set_populations: sync");
    }
    return LBM_OK;
}

lbm_status lbm_state_bytes(const lbm_lattice *h, size_t *bytes)
{
    if (!h || !bytes) return fail(LBM_EINVAL, "lbm_state_bytes: NULL argument");
    *bytes = lbm::state_bytes(h->phys.storage, h->phys.N);
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_lattice *h, void *dev_buf, size_t bytes)
{
    size_t need = 0;
    lbm_status st = lbm_state_bytes(h, &need);
    if (st != LBM_OK) return st;
    if (!dev_buf || bytes < need)
        return fail(LBM_EINVAL, "lbm_get_state: buffer of %zu bytes, need %zu", bytes, need);
    DeviceGuard g(h->device);
    CK(cudaMemcpyAsync(dev_buf, h->f[h->cur], need, cudaMemcpyDeviceToDevice, h->stream), "lbm_get_state");
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_lattice *h, const void *dev_buf, size_t bytes)
{
    size_t need = 0;
    lbm_status st = lbm_state_bytes(h, &need);
    if (st != LBM_OK) return st;
    if (!dev_buf || bytes < need)
        return fail(LBM_EINVAL, "lbm_set_state: buffer of %zu bytes, need %zu", bytes, need);
    DeviceGuard g(h->device);
    h->init_at_rest = 0;
    CK(cudaMemcpyAsync(h->f[h->cur], dev_buf, need, cudaMemcpyDeviceToDevice, h->stream), "lbm_set_state");
    return LBM_OK;
}

lbm_status lbm_step_count(const lbm_lattice *h, long *steps)
{
    if (!h || !steps) return fail(LBM_EINVAL, "lbm_step_count: NULL argument");
    *steps = h->steps;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_lattice *h)
{
    if (!h) return fail(LBM_EINVAL, "lbm_sync: NULL handle");
    DeviceGuard g(h->device);
    CK(cudaStreamSynchronize(h->stream), "lbm_sync");
    return LBM_OK;
}

lbm_status lbm_record(lbm_lattice *h, long n_steps, int ckpt_every)
{
    if (!h) return fail(LBM_EINVAL, "lbm_record: NULL handle");
    if (n_steps < 1 || ckpt_every < 1)
        return fail(LBM_EINVAL, "lbm_record: n_steps = %ld and ckpt_every = %d must be >= 1", n_steps, ckpt_every);
    DeviceGuard g(h->device);
    size_t sb = 0;
    lbm_state_bytes(h, &sb);
    const long nck = (n_steps + ckpt_every - 1) / ckpt_every;
    cudaFree(h->ckpt);
    h->ckpt = nullptr;
    h->rec_steps = 0;
    free_workspace(h);
    CK(cudaMalloc(&h->ckpt, sb * (size_t)nck), "lbm_record: checkpoint store");
    {
        const size_t N = (size_t)h->phys.N;
        const size_t rb = lbm::real_bytes(h->phys.storage);
        const size_t E = (size_t)(ckpt_every < n_steps ? ckpt_every : n_steps);
        CK(cudaMalloc(&h->ws_lam, rb * 2 * lbm::Q * N), "lbm_record: reverse-pass lambda");
        CK(cudaMalloc(&h->ws_lam_loc, rb * 2 * lbm::Q * N), "lbm_record: reverse-pass lambda_loc");
        CK(cudaMalloc(&h->ws_a, rb * 6 * N), "lbm_record: reverse-pass a");
        CK(cudaMalloc(&h->ws_d, rb * 4 * N), "lbm_record: reverse-pass D");
        // states 1 .. E-1 of a segment (state 0 is read from its checkpoint)
        CK(cudaMalloc(&h->ws_seg, sb * (size_t)(E > 1 ? E - 1 : 1)), "lbm_record: reverse-pass segment states");
        // per replayed step: the interaction sums (fused step, 6 N) or the
        // densities (two-kernel step, 2 N)
        CK(cudaMalloc(&h->ws_rseg, rb * (h->use_fused ? 6 : 2) * N * E), "lbm_record: reverse-pass segment sums");
        CK(cudaMalloc(&h->ws_io, sizeof(double) * 2 * N), "lbm_record: reverse-pass staging");
        CK(cudaMalloc((void **)&h->ws_part, sizeof(double) * 4 * lbm::adjoint_blocks(h->phys.storage)), "lbm_record: partials");
    }
    h->rec_at_rest = h->init_at_rest && h->steps == 0;
    for (long t = 0; t < n_steps; ++t) {
        if (t % ckpt_every == 0)
            CK(cudaMemcpyAsync((char *)h->ckpt + sb * (size_t)(t / ckpt_every), h->f[h->cur], sb,
                               cudaMemcpyDeviceToDevice, h->stream),
               "lbm_record: checkpoint");
        lbm_status st = lbm_step(h, 1);
        if (st != LBM_OK) return st;
    }
    CK(cudaStreamSynchronize(h->stream), "lbm_record: sync");
    h->rec_steps = n_steps;
    h->rec_every = ckpt_every;
    h->rec_nck = nck;
    return LBM_OK;
}

lbm_status lbm_adjoint(lbm_lattice *h, const double *dL_drho1, const double *dL_drho2, int on_device,
                       double *dL_drho1_0, double *dL_drho2_0, double dL_dparams[4])
{
    if (!h) return fail(LBM_EINVAL, "lbm_adjoint: NULL handle");
    if (h->rec_steps < 1 || !h->ckpt) return fail(LBM_EINVAL, "lbm_adjoint: no recorded run (call lbm_record)");
    if ((dL_drho1_0 || dL_drho2_0) && !h->rec_at_rest)
        return fail(LBM_ENOTSUP, "lbm_adjoint: initial-density gradients need a recording that starts at rest "
                                 "right after lbm_init_fields(u = NULL)");
    if ((long long)lbm::Q * h->phys.N > 0xffffffffLL)
        return fail(LBM_ENOTSUP, "lbm_adjoint: 19 N must stay below 2^32 (N <= 226,050,910 cells)");
    DeviceGuard g(h->device);
    const size_t N = (size_t)h->phys.N;
    const size_t rb = lbm::real_bytes(h->phys.storage);
    size_t sb = 0;
    lbm_state_bytes(h, &sb);
    const long E = h->rec_every;
    const int nb = lbm::adjoint_blocks(h->phys.storage);
    // working memory reserved by lbm_record
    void *lam = h->ws_lam, *lam_loc = h->ws_lam_loc, *abuf = h->ws_a, *seg = h->ws_seg, *io = h->ws_io;
    void *dbuf = h->ws_d, *rseg = h->ws_rseg;
    double *part = h->ws_part;
    if (!lam || !lam_loc || !abuf || !seg || !io || !dbuf || !rseg || !part)
        return fail(LBM_EINVAL, "lbm_adjoint: the reverse pass's working memory is missing (call lbm_record)");
    std::vector<double> parth((size_t)nb * 4);
    cudaError_t e;
    lbm_status st = LBM_OK;
    cudaStream_t cs = nullptr;   // capture stream of the segment graphs
    auto cleanup = [&]() {
        if (cs) cudaStreamDestroy(cs);
        cs = nullptr;
    };
#define CKA(expr, where)                                  \
    do {                                                  \
        e = (expr);                                       \
        if (e != cudaSuccess) { st = cuda_fail(e, where); cleanup(); return st; } \
    } while (0)
    CKA(cudaMemsetAsync(dbuf, 0, rb * 4 * N, h->stream), "lbm_adjoint: clear D");
    CKA(cudaMemsetAsync(part, 0, sizeof(double) * 4 * nb, h->stream), "lbm_adjoint: clear");
    double *io1 = (double *)io, *io2 = (double *)io + N;
    const double *g1 = dL_drho1, *g2 = dL_drho2;
    if (!on_device) {
        if (dL_drho1) CKA(cudaMemcpyAsync(io1, dL_drho1, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream), "lbm_adjoint: copy");
        if (dL_drho2) CKA(cudaMemcpyAsync(io2, dL_drho2, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream), "lbm_adjoint: copy");
        g1 = dL_drho1 ? io1 : nullptr;
        g2 = dL_drho2 ? io2 : nullptr;
    }
    CKA(lbm::launch_adjoint_seed(h->phys, g1, g2, 1, lam, h->stream), "lbm_adjoint: seed");
    void *d_cur = dbuf, *d_nxt = (char *)dbuf + rb * 2 * N;   // D^N = 0 (cleared above)
    const bool use_fused = h->use_fused;
    // One checkpoint segment of len steps on stream st: recompute its forward
    // states and their densities, then len reverse steps with the adjoint
    // fields ping-ponging from (la, da).
    // The fused replay keeps each step's interaction sums (6 N reals; for the
    // last state of a segment a sums-only launch); the two-kernel replay keeps
    // each step's densities (2 N reals; the last state's from a density pass).
    const size_t rstride = rb * (use_fused ? 6 : 2) * N;
    // One checkpoint segment of len steps on stream st: recompute its forward
    // states, then len reverse steps with the adjoint fields ping-ponging from
    // (la, da).
    // The segment's first state is read in place from the checkpoint store
    // (first); its later states go to the segment buffer (state t at slot t - 1).
    auto enqueue_segment = [&](cudaStream_t st, long len, const void *first, void *la, void *lb, void *da,
                               void *db) -> cudaError_t {
        auto state = [&](long t) -> void * {
            return t == 0 ? const_cast<void *>(first) : (void *)((char *)seg + sb * (size_t)(t - 1));
        };
        cudaError_t er = cudaSuccess;
        const long nrec = use_fused ? len : len - 1;
        for (long t = 0; t < nrec && er == cudaSuccess; ++t) {
            const void *fi = state(t);
            // the fused replay's last step only supplies the interaction sums
            void *fo = (use_fused && t == nrec - 1) ? nullptr : state(t + 1);
            void *rt = (char *)rseg + rstride * (size_t)t;
            er = use_fused ? lbm::launch_step_fused(h->phys, fi, fo, st, nullptr, rt)
                           : lbm::launch_step_split(h->phys, fi, fo, rt, st);
        }
        if (er == cudaSuccess && !use_fused)
            er = lbm::launch_density(h->phys, state(len - 1), (char *)rseg + rstride * (size_t)(len - 1), st);
        for (long t = len - 1; t >= 0 && er == cudaSuccess; --t) {
            const void *fn = state(t);
            const void *rn = (char *)rseg + rstride * (size_t)t;
            // step t reads (la, da) and writes (lb, db)
            er = lbm::launch_adjoint_step(h->phys, fn, rn, use_fused ? 1 : 0, la, da, lb, abuf, db, part, st);
            std::swap(la, lb);
            std::swap(da, db);
        }
        return er;
    };
    // A full segment replays a captured graph (one executable graph per
    // ping-pong parity of the adjoint fields): the same launches with one
    // launch instead of about 3E.  Each segment starts from its own
    // checkpoint, so its launches are captured afresh and applied to the
    // parity's executable graph (cudaGraphExecUpdate changes only later
    // launches; the host captures the next segment while the device runs the
    // current one).
    if (h->use_graphs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cs = nullptr;
        cudaGetLastError();
    }
    auto segment_graph = [&](int par, const void *first) -> cudaGraphExec_t {
        if (!cs || h->seg_graph_state[par] == -1) return nullptr;
        cudaGraph_t gr = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const cudaError_t er = enqueue_segment(cs, E, first, lam, lam_loc, d_cur, d_nxt);
            const cudaError_t ee = cudaStreamEndCapture(cs, &gr);
            ok = er == cudaSuccess && ee == cudaSuccess && gr;
        }
        if (ok && h->seg_graph_state[par] == 1) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(h->seg_graph[par], gr, &info) != cudaSuccess) {
                cudaGraphExecDestroy(h->seg_graph[par]);
                h->seg_graph[par] = nullptr;
                h->seg_graph_state[par] = 0;
            }
        }
        if (ok && h->seg_graph_state[par] == 0)
            h->seg_graph_state[par] = cudaGraphInstantiate(&h->seg_graph[par], gr, 0) == cudaSuccess ? 1 : -1;
        if (!ok && h->seg_graph_state[par] == 0) h->seg_graph_state[par] = -1;
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        return ok && h->seg_graph_state[par] == 1 ? h->seg_graph[par] : nullptr;
    };
    for (long k = h->rec_nck - 1; k >= 0; --k) {
        const long t0 = k * E;
        const long t1 = (t0 + E < h->rec_steps) ? t0 + E : h->rec_steps;
        const long len = t1 - t0;
        const void *first = (char *)h->ckpt + sb * (size_t)k;
        cudaGraphExec_t gx = len == E ? segment_graph(lam == h->ws_lam ? 0 : 1, first) : nullptr;
        if (gx) CKA(cudaGraphLaunch(gx, h->stream), "lbm_adjoint: segment graph");
        else CKA(enqueue_segment(h->stream, len, first, lam, lam_loc, d_cur, d_nxt), "lbm_adjoint: segment");
        if (len & 1) {
            std::swap(lam, lam_loc);
            std::swap(d_cur, d_nxt);
        }
    }
    if (dL_drho1_0 || dL_drho2_0) {
        double *o1 = on_device ? dL_drho1_0 : (dL_drho1_0 ? io1 : nullptr);
        double *o2 = on_device ? dL_drho2_0 : (dL_drho2_0 ? io2 : nullptr);
        CKA(lbm::launch_adjoint_rho0(h->phys, lam, d_cur, o1, o2, h->stream), "lbm_adjoint: rho0");
        if (!on_device) {
            if (dL_drho1_0) CKA(cudaMemcpyAsync(dL_drho1_0, io1, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream), "lbm_adjoint: copy out");
            if (dL_drho2_0) CKA(cudaMemcpyAsync(dL_drho2_0, io2, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream), "lbm_adjoint: copy out");
        }
    }
    CKA(cudaMemcpyAsync(parth.data(), part, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, h->stream),
        "lbm_adjoint: partials");
    CKA(cudaStreamSynchronize(h->stream), "lbm_adjoint: sync");
#undef CKA
    if (dL_dparams) {
        double acc[4] = {0, 0, 0, 0};
        for (int b = 0; b < nb; ++b)
            for (int q = 0; q < 4; ++q) acc[q] += parth[(size_t)b * 4 + q];
        for (int q = 0; q < 4; ++q) dL_dparams[q] = acc[q];
    }
    cleanup();
    return LBM_OK;
}

lbm_status lbm_step_noalloc(const lbm_params *pp, const void *f_in, void *f_out)
{
    if (!pp || !f_in || !f_out) return fail(LBM_EINVAL, "lbm_step_noalloc: NULL argument");
    if (f_in == f_out) return fail(LBM_EINVAL, "lbm_step_noalloc: f_in and f_out must be distinct buffers");
    const lbm_params &p = *pp;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1)
        return fail(LBM_EINVAL, "lbm_step_noalloc: sizes must be >= 1 (got %d x %d x %d)", p.nx, p.ny, p.nz);
    const long long N = (long long)p.nx * p.ny * p.nz;
    if (N > lbm::kNoallocMaxCells)
        return fail(LBM_EINVAL, "lbm_step_noalloc: %lld cells exceed the static scratch limit of %lld "
                                "(LBM_NOALLOC_MAX_CELLS); use lbm_create/lbm_step", N, lbm::kNoallocMaxCells);
    for (int a = 0; a < 2; ++a)
        if (!(p.tau[a] > 0.5) || !isfinite(p.tau[a]))
            return fail(LBM_EINVAL, "lbm_step_noalloc: tau[%d] = %g must be a finite value > 1/2", a, p.tau[a]);
    if (p.G[0][0] != 0.0 || p.G[1][1] != 0.0)
        return fail(LBM_ENOTSUP, "lbm_step_noalloc: G^{aa} must be 0");
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (!isfinite(p.G[a][b])) return fail(LBM_EINVAL, "lbm_step_noalloc: G must be finite");
    for (int d = 0; d < 3; ++d)
        if (!isfinite(p.g_ext[d])) return fail(LBM_EINVAL, "lbm_step_noalloc: g_ext must be finite");
    if (!isfinite(p.rho_s[0]) || !isfinite(p.rho_s[1]) || !isfinite(p.rho0_dev))
        return fail(LBM_EINVAL, "lbm_step_noalloc: rho_s and rho0_dev must be finite");
    if (p.storage < LBM_F64 || p.storage > LBM_BF16_REL)
        return fail(LBM_EINVAL, "lbm_step_noalloc: unknown storage %d", p.storage);
    if (p.storage != LBM_F16_DEV && p.storage != LBM_BF16_DEV && p.rho0_dev != 0.0)
        return fail(LBM_EINVAL, "lbm_step_noalloc: rho0_dev applies to the 16-bit deviation formats only");
    if (p.collision != LBM_BGK && p.collision != LBM_REGULARIZED && p.collision != LBM_REGULARIZED3)
        return fail(LBM_EINVAL, "lbm_step_noalloc: unknown collision %d", p.collision);
    if (p.wall_model != LBM_WALL_POTENTIAL && p.wall_model != LBM_WALL_MIRROR)
        return fail(LBM_EINVAL, "lbm_step_noalloc: unknown wall model %d", p.wall_model);
    if (p.forcing != LBM_FORCING_EDM && p.forcing != LBM_FORCING_GUO)
        return fail(LBM_EINVAL, "lbm_step_noalloc: unknown forcing %d", p.forcing);
    {
        // the step reads all of f_in while it writes f_out: the two states must not overlap
        const size_t sb = lbm::state_bytes(p.storage, N);
        const char *a0 = (const char *)f_in, *b0 = (const char *)f_out;
        if (a0 < b0 + sb && b0 < a0 + sb)
            return fail(LBM_EINVAL, "lbm_step_noalloc: f_in and f_out overlap (each state is %zu bytes)", sb);
    }
    for (int d = 0; d < 3; ++d)
        if (p.periodic[d] != 0 && p.periodic[d] != 1)
            return fail(LBM_EINVAL, "lbm_step_noalloc: periodic[%d] must be 0 or 1", d);
    if (!p.periodic[0] || !p.periodic[1])
        return fail(LBM_ENOTSUP, "lbm_step_noalloc: walls are supported along z only");
    lbm::HostPhys ph;
    ph.nx = p.nx; ph.ny = p.ny; ph.nz = p.nz; ph.N = N;
    ph.wall_z = p.periodic[2] ? 0 : 1;
    ph.wall_mirror = p.wall_model == LBM_WALL_MIRROR;
    ph.storage = p.storage;
    ph.collision = p.collision;
    ph.forcing = p.forcing;
    ph.tau[0] = p.tau[0]; ph.tau[1] = p.tau[1];
    ph.G12 = p.G[0][1]; ph.G21 = p.G[1][0];
    for (int d = 0; d < 3; ++d) ph.gext[d] = p.g_ext[d];
    ph.rho_s[0] = p.rho_s[0]; ph.rho_s[1] = p.rho_s[1];
    ph.rho0 = p.rho0_dev;
    ph.ref_off = (long long)lbm::ref_offset(p.storage, N);
    CK(lbm::launch_step_split_noalloc(ph, f_in, f_out, (cudaStream_t)p.stream), "lbm_step_noalloc");
    return LBM_OK;
}

const char *lbm_last_error(const lbm_lattice *)
{
    return g_err.c_str();
}

}  // extern "C"
