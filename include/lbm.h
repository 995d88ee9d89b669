/*
 * lbm.h - C ABI of the GB300 two-component D3Q19 Shan-Chen lattice Boltzmann
 * library (Otomo et al., "Studies of accurate multi-component lattice
 * Boltzmann models on benchmark cases required for engineering
 * applications", arXiv:1601.01237).
 *
 * One time step (Sec. 2, Eq. 1) advances the populations f_i^a(x, t) of the
 * two components a = 1, 2 on a D3Q19 lattice:
 *   1. moments rho^a = sum_i f_i^a, u = sum_a sum_i c_i f_i^a / rho (Eqs. 4-6);
 *   2. Shan-Chen interaction F^{ab} = G^{ab} rho^a sum_i w_i c_i rho^b(x + c_i)
 *      (Eq. 7), plus the wall interaction F_w^{ab} of Eq. 13 at solid
 *      neighbours, giving g^a = sum_b (F^{ab} + F_w^{ab}) / rho^a + g_ext;
 *   3. collision toward the third-order equilibrium f^eq(rho^a, u) of Eq. 3
 *      (T0 = 1/3): BGK (Eq. 2) or the regularized filter (Eqs. 10-11), plus the
 *      forcing term F_i^a = f^eq_i(rho^a, u + g^a) - f^eq_i(rho^a, u);
 *   4. streaming f_i^a(x + c_i, t + 1) = f*_i^a(x, t), periodic, or half-way
 *      bounce-back at solid walls (Sec. 4.1).
 *
 * Conventions shared by every call:
 *   - Fields are indexed [z][y][x] with x fastest; cell = (z*ny + y)*nx + x.
 *   - Every call returns an lbm_status; none exits or aborts.  On failure a
 *     message is available from lbm_last_error().
 *   - Pointers flagged `on_device` are CUDA device pointers on the device that
 *     was current at lbm_create; otherwise host pointers.  Caller-owned buffers
 *     are never retained: inputs are copied, outputs are written before the
 *     call returns (host) or in stream order (device).
 *   - All device work is issued on the lattice's stream (lbm_params.stream, or
 *     a stream the library creates when it is NULL).  Device outputs are valid
 *     once that stream has reached the call; host outputs are valid on return.
 *   - Errors of kernels already in flight surface at the next call that
 *     synchronizes (lbm_moments with host outputs, lbm_reduce, lbm_sync).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* invalid argument (sizes, tau <= 1/2, NULL pointer, ...) */
    LBM_ENOMEM = 2,    /* device allocation failed */
    LBM_ECUDA = 3,     /* CUDA runtime error (launch or asynchronous fault) */
    LBM_ENOTSUP = 4,   /* valid request this library does not implement */
    LBM_ENUMERIC = 5   /* non-finite or non-positive density met */
} lbm_status;

/* Population storage.  Arithmetic is FP64 for LBM_F64 and FP32 otherwise.
 * The *_DEV formats store the deviation f_i - w_i * rho0_dev in 16 bits.
 * The *_REL formats store the relative deviation f_i / (w_i rho~) - 1 in 16
 * bits, where rho~ is the density (of the population's own component), at
 * the step that produced the population, of the cell that reads it next;
 * every cell keeps its own pair (rho~1, rho~2) in FP32 beside the
 * populations (8 more bytes per cell), so that both phases of a
 * phase-separated state keep the full 16-bit precision (rho0_dev must be 0).
 * None of the 16-bit codecs comes from the paper. */
typedef enum {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F16_DEV = 2,
    LBM_BF16_DEV = 3,
    LBM_F16_REL = 4,
    LBM_BF16_REL = 5
} lbm_storage;

typedef enum {
    LBM_BGK = 0,          /* Eq. 2 */
    LBM_REGULARIZED = 1,  /* Eqs. 10-11, second-order Hermite projection */
    LBM_REGULARIZED3 = 2  /* Eqs. 10-11 keeping also the third-order
                             non-equilibrium moments ("energy flux", Sec. 2):
                             f^neq is the w-weighted projection of
                             (f - f^eq) / w_i onto the second- and
                             third-order Hermite polynomials that D3Q19
                             carries (6 + 6 of them) */
} lbm_collision;

/* The forcing term of Eq. 1 (Sec. 2 cites the scheme without printing it). */
typedef enum {
    LBM_FORCING_EDM = 0,  /* exact difference of equilibria:
                             F_i = f^eq_i(rho^a, u + g^a) - f^eq_i(rho^a, u), f^eq at
                             the mixture velocity u of Eq. 6 */
    LBM_FORCING_GUO = 1   /* Guo, Zheng & Shi (2002) per component with the common
                             equilibrium velocity u* = u + g/2 of Eqs. 8-9:
                             F_i = (1 - 1/(2 tau)) w_i [(c_i - u*)/T0 + (c_i.u*) c_i / T0^2]
                             . rho^a g^a for BGK; the regularized filter keeps
                             f^eq(u*) + (1 - 1/tau) P[f - f^eq(u*) + F/2] + F/2 with
                             F the bracket without the tau factor */
} lbm_forcing;

/* Density a solid site presents to the interaction sum of Eq. 13. */
typedef enum {
    LBM_WALL_POTENTIAL = 0, /* rho'_b = rho_s^b (point-wise wall potential, Sec. 4) */
    LBM_WALL_MIRROR = 1     /* rho'_b = rho_b(mirror cell) + rho_s^b: zero normal
                               derivative as Eq. 13 asks (modified model, Sec. 4.1) */
} lbm_wall_model;

typedef struct {
    int nx, ny, nz;        /* lattice cells along x, y, z (each >= 1) */
    int periodic[3];       /* 1 = periodic.  periodic[0] and periodic[1] must be 1;
                              periodic[2] = 0 puts half-way bounce-back walls at
                              z = -1/2 and z = nz - 1/2 */
    double tau[2];         /* relaxation times tau_1, tau_2 (Eq. 2), each > 1/2 */
    double G[2][2];        /* G^{ab} of Eq. 7, signed exactly as printed there
                              (repulsion between components is G < 0).
                              G[0][0] and G[1][1] must be 0 (Sec. 2). */
    double g_ext[3];       /* body acceleration added to every g^a */
    double rho_s[2];       /* wall potential rho_s^a (Sec. 4.2) */
    double rho0_dev;       /* reference density of the *_DEV storage formats */
    int storage;           /* lbm_storage */
    int collision;         /* lbm_collision */
    int wall_model;        /* lbm_wall_model (used only when periodic[2] == 0) */
    void *stream;          /* cudaStream_t to issue work on; NULL = library-owned stream */
    int forcing;           /* lbm_forcing */
} lbm_params;

typedef struct lbm_lattice lbm_lattice;   /* opaque handle */

/* The library's D3Q19 direction order (the lattice of Sec. 2): c[i] and w[i].
 * Populations passed through lbm_get_populations / lbm_set_populations use it.
 * Either pointer may be NULL. */
lbm_status lbm_lattice_dirs(int c[19][3], double w[19]);

/* Validate *params, allocate device storage for two population copies and the
 * density scratch, and return a handle in *out.  Errors: LBM_EINVAL (bad
 * sizes, tau <= 1/2, NULL pointers, F64 with rho0_dev != 0), LBM_ENOTSUP
 * (non-zero G^{aa}, x/y walls), LBM_ENOMEM, LBM_ECUDA.  The handle owns its
 * device memory until lbm_destroy. */
lbm_status lbm_create(const lbm_params *params, lbm_lattice **out);

/* Initial state f_i^a(x, 0) = f^eq_i(rho^a_0(x), u_0(x)) (Eq. 3).  rho1, rho2:
 * N = nx*ny*nz doubles each; u: 3N doubles [cell][3] or NULL for u = 0.
 * Host or device pointers (on_device); contents are copied, host fields
 * through the lattice's second population copy (no allocation), and the call
 * synchronizes before it returns when they are host pointers, so the caller
 * may reuse them.  Resets the step counter to 0.  Errors: LBM_EINVAL,
 * LBM_ECUDA. */
lbm_status lbm_init_fields(lbm_lattice *h, const double *rho1, const double *rho2,
                           const double *u, int on_device);

/* Advance n_steps >= 0 full time steps (moments, interaction force, collision
 * with forcing, streaming; Sec. 2 and Eq. 1 or Eq. 10).  Asynchronous on the
 * lattice's stream.  Errors: LBM_EINVAL (n_steps < 0), LBM_ECUDA. */
lbm_status lbm_step(lbm_lattice *h, long n_steps);

/* lbm_step with per-kernel timing: advances n_steps > 0 steps exactly as
 * lbm_step does, recording a CUDA event pair around every kernel launch on the
 * lattice's stream, then synchronizes.  kernel_ms[k] receives the total device
 * time of kernel kind k over the n_steps, launches[k] its launch count, and
 * names[k] (static strings) its name, for k < *n_kinds <= 4.  Used by the
 * benchmark for per-launch durations.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_step_timed(lbm_lattice *h, long n_steps, double kernel_ms[4], long launches[4],
                          const char *names[4], int *n_kinds);

/* Output fields of the current state: rho^1, rho^2 (N values each) and the
 * velocity u_F = u + g/2 (Eqs. 8-9; 3N values [cell][3]).  Element type is
 * double when out_f64 != 0, else float.  Any output pointer may be NULL.
 * Host outputs synchronize the stream; device outputs are stream-ordered. */
lbm_status lbm_moments(lbm_lattice *h, int out_f64, void *rho1, void *rho2, void *uF,
                       int on_device);

/* FP64 reductions of the current state into out[6]:
 *   out[0] = sum rho^1, out[1] = sum rho^2,
 *   out[2..4] = sum rho u_F (total momentum), out[5] = max |u_F|.
 * Synchronizes the stream.  Returns LBM_ENUMERIC if a density is non-finite
 * or not positive. */
lbm_status lbm_reduce(lbm_lattice *h, double out[6]);

/* Pressure jump across a droplet interface (Young-Laplace, Eq. 12), reduced
 * in FP64 on the GPU.  The pressure is the bulk pressure of the Eq. 7 force,
 * p = T0 (rho^1 + rho^2) - G^{12} T0 rho^1 rho^2 (T0 = 1/3; a reading: the
 * paper does not define p).  out[0] = mean p over cells with distance
 * < r_in from center[3] (x, y, z lattice coordinates; minimum image along
 * periodic axes), out[1] = mean p over cells with distance > r_out, out[2] =
 * out[0] - out[1].  Synchronizes.  Errors: LBM_EINVAL (NULL, r_in <= 0,
 * an empty region), LBM_ECUDA. */
lbm_status lbm_pressure_jump(lbm_lattice *h, const double center[3], double r_in, double r_out, double out[3]);

/* Droplet statistics of component 1 for the wall cases (Sec. 4.2), FP64 on
 * the GPU.  Droplet = cells with rho^1 > threshold.  out[0] = droplet volume
 * (cells), out[1..3] = its centre of mass (mean x, y, z relative to origin[3],
 * minimum image along periodic axes), out[4] = mass of component 1 inside it,
 * out[5] = mean rho^1 of the wall layer z = 0 (with a solid mask: the fluid
 * cells next to a solid site) outside the droplet (thin-film density),
 * out[6] = number of those cells.  Synchronizes.  Errors:
 * LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_droplet_stats(lbm_lattice *h, double threshold, const double origin[3], double out[7]);

/* Staircase walls of any shape (the inclined walls of Sec. 4.2): solid[cell]
 * != 0 marks a solid site, N bytes in [z][y][x] order, host (on_device = 0)
 * or device memory, copied.  Every link into a solid site is a half-way
 * bounce-back link; solid sites hold no fluid (their populations, densities
 * and velocities read as 0); in Eq. 13 a solid site presents the w-weighted
 * mean of rho^b over its fluid neighbours plus rho_s^b (LBM_WALL_MIRROR) or
 * rho_s^b alone (LBM_WALL_POTENTIAL).  NULL removes the mask.  A lattice
 * with a mask steps with the fused step (the FP32 and 16-bit formats) or
 * the two-kernel step (LBM_F64); under the mirror model the fused step first
 * refreshes the wall densities of the solid sites next to fluid with two
 * small kernels over those sites and their fluid neighbours.  lbm_record and
 * lbm_adjoint take the mask (bounce-back links and, for the mirror model,
 * the dependence of the wall densities on the fluid densities).
 * lbm_pressure_jump and lbm_droplet_stats leave solid sites out, and the
 * thin-film layer of lbm_droplet_stats is then the fluid cells next to a
 * solid site.  Set the mask before lbm_init_fields (a state set earlier
 * keeps the populations of the new solid sites, which are never read).  The
 * library keeps on the device, until the mask is removed or the lattice
 * destroyed: the mask, one 32-bit word of link flags per cell (bit i: the
 * site x - c_i is solid, bit 0: x itself), a pair of FP32 wall densities per
 * cell, and the lists of the solid sites next to fluid and of the fluid
 * cells next to a solid site (13 bytes per cell and 4 per listed cell).
 * Drops the lattice's recording.  Synchronizes.  Errors: LBM_EINVAL (NULL handle),
 * LBM_ENOTSUP (lattice with walls along z), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_set_solid(lbm_lattice *h, const unsigned char *solid, int on_device);

/* Copy the populations f_i^a(x, t) of the current state, as doubles laid out
 * [a][i][z][y][x] in the lbm_lattice_dirs order (2*19*N values), to or from a
 * caller buffer (host or device).  Used for checkpoints and for population-level
 * checks; set also resets nothing else (the step counter is kept). */
lbm_status lbm_get_populations(lbm_lattice *h, double *out, int on_device);
lbm_status lbm_set_populations(lbm_lattice *h, const double *in, int on_device);

/* Raw state (the storage-format populations) for fast checkpoints:
 * lbm_state_bytes gives the size; get/set copy it to or from a
 * caller device buffer of at least that many bytes.  Layout: population i
 * of component a at cell c (x fastest) is element 2 (i N + c) + a in the
 * storage type (the two components of a direction side by side); the values
 * are the post-collision populations at their origin cell.  The *_REL
 * formats follow them, at the population bytes rounded up to a multiple of
 * 256, with the N reference pairs (rho~1, rho~2) as FP32 (cell c at pair c). */
lbm_status lbm_state_bytes(const lbm_lattice *h, size_t *bytes);
lbm_status lbm_get_state(lbm_lattice *h, void *dev_buf, size_t bytes);
lbm_status lbm_set_state(lbm_lattice *h, const void *dev_buf, size_t bytes);

/* Number of time steps taken since the last lbm_init_fields. */
lbm_status lbm_step_count(const lbm_lattice *h, long *steps);

/* Wait for all work issued on the lattice's stream; reports asynchronous
 * errors as LBM_ECUDA. */
lbm_status lbm_sync(lbm_lattice *h);

/* Differentiation (reverse mode).  The paper has no adjoint; these calls give
 * gradients of a loss L(rho^1_N, rho^2_N) of the final densities with respect
 * to the initial densities, G^{12}, G^{21}, tau_1 and tau_2, by a hand-written
 * reverse pass through the update of Sec. 2 (Eqs. 1-7, 10-11, 13), for either
 * forcing reading, every collision operator, periodic lattices, z walls and
 * solid masks.
 *
 * lbm_record runs n_steps >= 1 forward exactly as lbm_step does and keeps the
 * raw state every ckpt_every >= 1 steps (a library-owned checkpoint store of
 * ceil(n_steps / ckpt_every) states), and reserves the working memory of the
 * reverse pass (adjoint fields of 2 x 19 values per cell, one checkpoint
 * segment of states and of their densities); both are held until the next
 * lbm_record or lbm_destroy, so that lbm_adjoint allocates nothing.
 * Synchronizes.  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_record(lbm_lattice *h, long n_steps, int ckpt_every);

/* Reverse pass over the last lbm_record.  Inputs dL_drho1, dL_drho2: N values
 * each (double), dL/drho^a of the recorded run's final state; either may be
 * NULL (zero).  Outputs (each may be NULL): dL_drho1_0, dL_drho2_0 (N doubles),
 * the gradient with respect to the initial densities of a run started by
 * lbm_init_fields with u = NULL (f = w_i rho at rest); dL_dparams[4] (host) =
 * dL/dG^{12}, dL/dG^{21}, dL/dtau_1, dL/dtau_2 (for a tied G^{12} = G^{21},
 * sum the first two).  All array pointers are host (on_device = 0) or device
 * (on_device = 1) memory.  The forward states of each checkpoint segment are
 * recomputed (time-checkpointing) in the working memory that lbm_record
 * reserved; the call may be repeated with other loss gradients.  Leaves the
 * lattice state at the end of the recorded run.
 * Synchronizes.  Errors: LBM_EINVAL (no recording), LBM_ENOTSUP
 * (initial-density gradient requested for a recording that did not start at
 * rest from lbm_init_fields, or a lattice with 19 N >= 2^32 cells),
 * LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_adjoint(lbm_lattice *h, const double *dL_drho1, const double *dL_drho2, int on_device,
                       double *dL_drho1_0, double *dL_drho2_0, double dL_dparams[4]);

/* Largest lattice (nx*ny*nz cells) that lbm_step_noalloc accepts: 128^3. */
#define LBM_NOALLOC_MAX_CELLS 2097152L

/* One time step for callers that cannot allocate device memory.  The paper
 * has no counterpart to this call; it exists for integrations where the
 * caller owns every device buffer and cudaMalloc is not allowed at step time
 * (for example host code running under a memory-pool policy that forbids
 * allocation, or a real-time loop that must not take the allocator's locks).
 *
 * It advances the state in f_in by one step into f_out with the two-kernel
 * step (density pass, then force + collision + streaming).  f_in and f_out are
 * caller-owned device buffers in the raw state format (the layout
 * lbm_get_state writes; lbm_state_bytes of a lattice with the same params)
 * that must not overlap (LBM_EINVAL otherwise).
 * *params is validated as by lbm_create, except that params->stream = NULL
 * means the default stream.  No handle is created and nothing is allocated:
 * the density scratch is a static device array of 32 MiB built into the
 * library, held on every device that loads it until the process exits.
 *
 * Limits and sharing: lattices above LBM_NOALLOC_MAX_CELLS cells are rejected
 * with LBM_EINVAL.  The scratch is written in full by the density pass before
 * the collision reads it, so nothing needs clearing between calls, but every
 * call shares it: calls whose work overlaps on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  The first call on
 * a device looks up the scratch's device address (set-up); with lazy module
 * loading that lookup also loads the library's device code and makes the
 * 32 MiB array resident on the device, which is an allocation by the CUDA
 * runtime.  A caller whose policy forbids any allocation while stepping, or
 * that captures streams, makes that first call during set-up.  Asynchronous
 * on the stream; errors: LBM_EINVAL, LBM_ENOTSUP, LBM_ECUDA. */
lbm_status lbm_step_noalloc(const lbm_params *params, const void *f_in, void *f_out);

/* Release every resource of the handle.  NULL-safe. */
void lbm_destroy(lbm_lattice *h);

/* Message of the last failure on this thread (empty string if none).  The
 * handle may be NULL. */
const char *lbm_last_error(const lbm_lattice *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
