// Internal interface between the C ABI (lbm_api.cu) and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/lbm.h"

namespace lbm {

// Launch geometry and physics of one lattice, in host form.
struct HostPhys {
    int nx, ny, nz;
    long long N;
    int wall_z;
    int wall_mirror;
    int storage;
    int collision;
    int forcing = 0;   // lbm_forcing (0 exact difference, 1 Guo)
    double tau[2];
    double G12, G21;
    double gext[3];
    double rho_s[2];
    double rho0;
    // N flags on the device, 1 = solid site (staircase walls); nullptr = none.
    // Only the two-kernel step and its density, output and reduction kernels
    // take a mask.
    const unsigned char *solid = nullptr;
    // N words of link flags derived from the mask: bit i set when the pull
    // source x - c_i of cell x is a solid site (bit 0: x itself is solid;
    // launch_link_flags)
    const unsigned *links = nullptr;
    // *_REL formats: byte offset of the per-cell reference densities from the
    // base of a state (see state_bytes); 0 otherwise
    long long ref_off = 0;
    // Fused step under a mask: N pairs (rho^1, rho^2) holding, at each solid
    // site, the density it presents to Eq. 13 (rho_s; for the mirror model
    // the sites listed in bsolid are refreshed before every fused step, through
    // the entries of the fluid cells listed in bfluid).  nullptr = no mask.
    const float *wall_rho = nullptr;
    const unsigned *bfluid = nullptr;   // fluid cells with a solid neighbour
    const unsigned *bsolid = nullptr;   // solid sites with a fluid neighbour
    long long n_bfluid = 0, n_bsolid = 0;
};

// Populations are stored as 2*19*N values of the storage type, laid out
// [a][i][cell], holding the post-collision values f*_i^a at their origin cell
// ("pull" streaming: f_i^a(x, t) = f*_i^a(x - c_i, t - 1), or the reversed
// population of x itself when x - c_i is a wall site).

// One full time step with the two-kernel design: density pass into rho
// (scratch, 2*N arithmetic values), then force + collision + streaming from
// f_in into f_out.
// ev (optional, 3 events): recorded before the density pass, between the
// passes and after the collision pass.
cudaError_t launch_step_split(const HostPhys &p, const void *f_in, void *f_out, void *rho,
                              cudaStream_t s, cudaEvent_t *ev = nullptr);

// One full time step with the fused single-pass kernel (no scratch).
// ev (optional, 2 events): recorded before and after the launch.
// s_out (optional, 6*N FP32 values, [3 b + d][cell]): receives the step's
// interaction sums S^b_d of Eq. 7 (the replay of the reverse pass uses them);
// with f_out == nullptr the launch computes and stores the sums alone.
cudaError_t launch_step_fused(const HostPhys &p, const void *f_in, void *f_out, cudaStream_t s,
                              cudaEvent_t *ev = nullptr, void *s_out = nullptr);
bool fused_supported(const HostPhys &p);
// Planes per CTA of the fused step for a lattice of cols = ceil(nx/32) *
// ceil(ny/8) tile columns and nz planes on a device with sms SMs.
constexpr int kPlanesMax = 64, kPlanesMin = 8;
int fused_planes(long long cols, int nz, int sms);

// Mask set-up for the fused step: wall_rho = rho_s at every solid site, and
// the counts (lists == nullptr) or the lists themselves of the boundary cells
// of the mirror model (fluid cells with a solid neighbour, solid sites with a
// fluid one); counts[0..1] must be zero on entry.
cudaError_t launch_mask_setup(const HostPhys &h, const unsigned char *solid, float *wall_rho, unsigned *bfluid,
                              unsigned *bsolid, unsigned long long *counts, cudaStream_t s);

// State set-up: populations from (rho1, rho2, u) via f^eq (u may be NULL),
// or from explicit populations f[a][i][cell] in library order (doubles).
// scratch (may be NULL): a second state copy, overwritten by the rest values
// of a state at rest (u == NULL).
cudaError_t launch_init_feq(const HostPhys &p, const double *rho1, const double *rho2,
                            const double *u, void *f, void *scratch, cudaStream_t s);
cudaError_t launch_set_populations(const HostPhys &p, const double *src, void *f, cudaStream_t s);
cudaError_t launch_get_populations(const HostPhys &p, const void *f, double *dst, cudaStream_t s);

// Output fields (rho1, rho2, u_F), each pointer optional; out_f64 selects the
// element type.  Uses rho (scratch) for the density pass.
cudaError_t launch_moments(const HostPhys &p, const void *f, void *rho, int out_f64,
                           void *rho1, void *rho2, void *uF, cudaStream_t s);

// FP64 reduction partials: nblocks x 8 doubles
// (mass1, mass2, px, py, pz, max|uF|, bad-density count, unused).
int reduce_blocks();
cudaError_t launch_reduce(const HostPhys &p, const void *f, void *rho, double *partials,
                          cudaStream_t s);

// Two-kernel step whose density scratch is the library's static device array
// (no allocation).  N must not exceed kNoallocMaxCells.
constexpr long long kNoallocMaxCells = 2097152;   // 128^3
cudaError_t launch_step_split_noalloc(const HostPhys &p, const void *f_in, void *f_out, cudaStream_t s);

// Reverse (adjoint) step n: from lambda_loc^{n+1} (2*19*N reals) and D^{n+1}
// (2*N reals) and the forward state f^n (raw state) with either its densities
// (rho, 2*N reals) or, when rho_is_sums, its interaction sums (rho, 6*N reals
// [3 b + d][cell], as written by launch_step_fused's s_out), writes
// lambda_loc^n, a^n (6*N reals, scratch) and D^n; partials
// (adjoint_blocks(storage) x 4 doubles: dG12, dG21, dtau1, dtau2) accumulate.
// lambda^n = lambda_loc^n + D^n of the population's component.
int adjoint_blocks(int storage);
cudaError_t launch_adjoint_step(const HostPhys &p, const void *f, const void *rho, int rho_is_sums,
                                const void *lam_next, const void *Dn, void *lam_loc, void *a, void *Dout,
                                double *partials, cudaStream_t s);
// lambda_loc^N_i = dL/drho^a of the component of i (g1/g2 may be NULL).
cudaError_t launch_adjoint_seed(const HostPhys &p, const void *g1, const void *g2, int g_f64, void *lam,
                                cudaStream_t s);
// dL/drho^a_0 = sum_i w_i lambda^0_i for an initial state f^eq(rho_0, u = 0).
cudaError_t launch_adjoint_rho0(const HostPhys &p, const void *lam, const void *D, double *g1, double *g2,
                                cudaStream_t s);
// density pass only (rho = sum_i f_i, pull-gathered) into rho
cudaError_t launch_density(const HostPhys &p, const void *f, void *rho, cudaStream_t s);

// FP64 diagnostics over the density fields in rho (diag_blocks() x
// diag_slots() partial doubles).
int diag_blocks();
int diag_slots();
cudaError_t launch_pressure(const HostPhys &h, const void *rho, const double center[3], double r_in, double r_out,
                            double *partials, cudaStream_t s);
cudaError_t launch_droplet(const HostPhys &h, const void *rho, double threshold, const double origin[3],
                           double *partials, cudaStream_t s);

// Link flags of a solid mask (N words, see HostPhys::links).
cudaError_t launch_link_flags(const HostPhys &p, const unsigned char *solid, unsigned *links, cudaStream_t s);

// Number of SMs of the current device, looked up once per device (every
// device of the process has its own entry; safe to call from several host
// threads).
int current_device_sms();

size_t storage_bytes(int storage);   // bytes per stored population value
// One raw state: the 2*19*N populations, and for the *_REL formats the N
// reference-density pairs (float2) behind them at ref_offset (the population
// bytes rounded up to 256).
bool storage_is_rel(int storage);
size_t ref_offset(int storage, long long N);
size_t state_bytes(int storage, long long N);
size_t real_bytes(int storage);      // bytes per arithmetic value

}  // namespace lbm
