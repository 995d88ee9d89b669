/*
 * FP64 CPU oracle for the two-component D3Q19 Shan-Chen lattice Boltzmann
 * update of Otomo et al., "Studies of accurate multi-component lattice
 * Boltzmann models on benchmark cases required for engineering
 * applications" (arXiv:1601.01237).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of the method that the CUDA library is checked against.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine is a plain loop over cells in the order the paper states the
 * update (Sec. 2): moments (Eqs. 4-6) -> Shan-Chen force (Eq. 7) and the
 * wall interaction (Eq. 13) -> collision toward the third-order equilibrium
 * (Eq. 3) with BGK (Eq. 2) or the regularized filter (Eqs. 10-11) plus the
 * forcing term -> streaming (left-hand side of Eq. 1).  No tiling, fusion or
 * reordering.  With OpenMP, each pass runs its outer loop over cells (or z
 * planes) on several threads; no pass reduces across cells, so the result
 * does not depend on the thread count.
 *
 * Readings of passages the paper leaves open:
 *  - D3Q19 velocities and weights are not printed (Sec. 2 only names the
 *    set): the textbook set, rest 1/3, six axis links 1/18, twelve face
 *    diagonals 1/36.  Here they are generated from their definition
 *    (all c in {-1,0,1}^3 with |c|^2 <= 2, weight by |c|^2).
 *  - The forcing term cites a reference that is not available (Sec. 2): the
 *    exact-difference form F_i = f^eq_i(rho^a, u + g^a) - f^eq_i(rho^a, u),
 *    which makes the velocity averaged over pre- and post-collision equal to
 *    u + g/2 as Eq. 8 states (forcing = 0).  The second reading (forcing = 1)
 *    is the scheme of Guo, Zheng & Shi, Phys. Rev. E 65, 046308 (2002),
 *    applied per component with one common equilibrium velocity
 *    u* = u + g/2 (Eqs. 8-9): f^eq(rho^a, u*), forcing term
 *    (1 - 1/(2 tau)) w_i [(c_i - u*)/T0 + (c_i.u*) c_i / T0^2] . rho^a g^a for
 *    BGK; for the regularized filter the same scheme written as
 *    f* = f^eq + (1 - 1/tau) P[f - f^eq + F/2] + F/2, P the Hermite
 *    projection of Eq. 11 (so Pi^neq gains (u* F + F u*) / 2).
 *  - The regularized non-equilibrium part (Eq. 11) is the second-order Hermite
 *    projection w_i/(2 T0^2) Q_i : Pi^neq, Q_i = c_i c_i - T0 I, with Pi^neq
 *    from the pre-collision populations and f^eq(rho^a, u).  Sec. 2 also
 *    keeps third-order non-equilibrium moments ("the energy flux"); the
 *    collision = 2 variant adds the orthogonal projection (weighted by w_i)
 *    of (f - f^eq) / w_i onto the span of the third-order Hermite polynomials
 *    H_abc(c_i) = c_a c_b c_c - T0 (c_a d_bc + c_b d_ac + c_c d_ab) evaluated
 *    on the lattice (every third-order moment the lattice can carry).
 *  - Walls (Sec. 4.1): half-way bounce-back; a solid site's density in
 *    Eq. 13 is rho'_b = rho_b(mirror cell) + rho_s^b for the modified model
 *    (zero normal derivative) or rho'_b = rho_s^b for the original
 *    point-wise wall potential.
 *  - Staircase walls of any shape (the inclined walls of Sec. 4.2) are a mask
 *    of solid sites: half-way bounce-back on every link into a solid site,
 *    and a solid site's density in Eq. 13 is the w-weighted mean of its
 *    fluid neighbours' densities (plus rho_s) for the modified model, rho_s
 *    for the original one.
 *  - G is taken literally as printed in Eq. 7 (signed; a repulsive
 *    interaction has G < 0).  The wall force of Eq. 13 uses the same G^{ab}.
 *
 * Layout: f[(a*19 + i)*N + cell], cell = (z*ny + y)*nx + x, x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define T0 (1.0 / 3.0)

typedef struct {
    int nx, ny, nz;
    int periodic[3];   /* 1 = periodic, 0 = solid half-way walls at both ends */
    double tau[2];
    double G[2][2];
    double g_ext[3];   /* body acceleration added to every component */
    double rho_s[2];   /* wall potential of each component */
    int collision;     /* 0 = BGK (Eq. 2), 1 = regularized filter (Eqs. 10-11),
                          2 = the same with third-order moments kept */
    int wall_model;    /* 0 = point-wise wall potential, 1 = mirrored rho' + rho_s */
    const unsigned char *solid;  /* N flags, 1 = solid site inside the lattice
                                    (staircase walls of any shape); NULL = none */
    int forcing;       /* 0 = exact difference of equilibria, 1 = Guo, Zheng &
                          Shi (2002) with the half-force velocity shift */
} oracle_params;

/* Lattices below this many cells run every pass on one thread (a parallel
 * region costs more than their work). */
#define OMP_BIG(p) ((long)(p)->nx * (p)->ny * (p)->nz > 32768L)

static int C[Q][3];
static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;
/* Orthonormal basis (inner product sum_i w_i g_i h_i) of the span of the
 * third-order Hermite polynomials on the lattice, N3 vectors. */
static double E3[10][Q];
static int N3 = 0;

/* D3Q19 (Sec. 2): enumerate every c in {-1,0,1}^3 with |c|^2 <= 2. */
static void build_lattice(void)
{
    if (lattice_ready) return;
    int n = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int m = cx * cx + cy * cy + cz * cz;
                if (m > 2) continue;
                C[n][0] = cx; C[n][1] = cy; C[n][2] = cz;
                W[n] = (m == 0) ? 1.0 / 3.0 : (m == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                ++n;
            }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2])
                OPP[i] = j;
    /* Gram-Schmidt over H_abc, a <= b <= c; vectors that vanish on the
     * lattice or depend on earlier ones are dropped */
    N3 = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            for (int c = b; c < 3; ++c) {
                double v[Q];
                for (int i = 0; i < Q; ++i)
                    v[i] = C[i][a] * C[i][b] * C[i][c] -
                           T0 * (C[i][a] * (b == c) + C[i][b] * (a == c) + C[i][c] * (a == b));
                for (int k = 0; k < N3; ++k) {
                    double d = 0.0;
                    for (int i = 0; i < Q; ++i) d += W[i] * v[i] * E3[k][i];
                    for (int i = 0; i < Q; ++i) v[i] -= d * E3[k][i];
                }
                double nn = 0.0;
                for (int i = 0; i < Q; ++i) nn += W[i] * v[i] * v[i];
                if (nn < 1e-24) continue;
                for (int i = 0; i < Q; ++i) E3[N3][i] = v[i] / sqrt(nn);
                ++N3;
            }
    lattice_ready = 1;
}

void oracle_lattice(int c[Q][3], double w[Q])
{
    build_lattice();
    for (int i = 0; i < Q; ++i) {
        c[i][0] = C[i][0]; c[i][1] = C[i][1]; c[i][2] = C[i][2];
        w[i] = W[i];
    }
}

/* Third-order equilibrium, Eq. 3, term by term as printed. */
void oracle_feq(double rho, const double u[3], double feq[Q])
{
    build_lattice();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        feq[i] = rho * W[i] * (1.0
                               + cu / T0
                               + (cu * cu) / (2.0 * T0 * T0)
                               - uu / (2.0 * T0)
                               + (cu * cu * cu) / (6.0 * T0 * T0 * T0)
                               - cu * uu / (2.0 * T0 * T0));
    }
}

static long cell_index(const oracle_params *p, int x, int y, int z)
{
    return ((long)z * p->ny + y) * p->nx + x;
}

static int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* Is lattice site (x,y,z), inside the lattice, flagged solid in the mask? */
static int mask_solid(const oracle_params *p, int x, int y, int z)
{
    return p->solid && p->solid[cell_index(p, x, y, z)];
}

/* Is lattice site (x,y,z) (possibly out of range) a solid wall site: beyond a
 * non-periodic end, or (after periodic wrap) flagged in the mask? */
static int is_solid(const oracle_params *p, int x, int y, int z)
{
    if (!p->periodic[0] && (x < 0 || x >= p->nx)) return 1;
    if (!p->periodic[1] && (y < 0 || y >= p->ny)) return 1;
    if (!p->periodic[2] && (z < 0 || z >= p->nz)) return 1;
    return mask_solid(p, wrap(x, p->nx), wrap(y, p->ny), wrap(z, p->nz));
}

/* Eqs. 4-6: rho^a = sum_i f_i^a; rho = sum_a rho^a;
 * u = sum_a sum_i c_i f_i^a / rho (one mixture velocity). */
void oracle_moments_raw(const oracle_params *p, const double *f,
                        double *rho1, double *rho2, double *u)
{
    build_lattice();
    long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
    for (long s = 0; s < N; ++s) {
        if (p->solid && p->solid[s]) {   /* no fluid at a solid site */
            rho1[s] = rho2[s] = 0.0;
            u[3 * s] = u[3 * s + 1] = u[3 * s + 2] = 0.0;
            continue;
        }
        double r[2] = {0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 2; ++a)
            for (int i = 0; i < Q; ++i) {
                double fi = f[((long)a * Q + i) * N + s];
                r[a] += fi;
                j[0] += C[i][0] * fi;
                j[1] += C[i][1] * fi;
                j[2] += C[i][2] * fi;
            }
        rho1[s] = r[0];
        rho2[s] = r[1];
        double rho = r[0] + r[1];
        u[3 * s + 0] = j[0] / rho;
        u[3 * s + 1] = j[1] / rho;
        u[3 * s + 2] = j[2] / rho;
    }
}

/* Density a solid site presents to the interaction sum (Eq. 13): the
 * modified model mirrors the adjacent fluid cell across the wall (zero
 * normal derivative) and adds rho_s; the original model uses rho_s alone.
 * A solid site of the mask has no single mirror cell: its density is the
 * mean of rho_b over its fluid neighbours, weighted by w_i (a volumetric
 * construction whose normal derivative vanishes for fields that vary along
 * the wall normal only), plus rho_s. */
static double wall_density(const oracle_params *p, const double *rho_b, double rho_s,
                           int x, int y, int z)
{
    if (p->wall_model == 0) return rho_s;
    {
        int in = (p->periodic[0] || (x >= 0 && x < p->nx)) && (p->periodic[1] || (y >= 0 && y < p->ny)) &&
                 (p->periodic[2] || (z >= 0 && z < p->nz));
        if (in && mask_solid(p, wrap(x, p->nx), wrap(y, p->ny), wrap(z, p->nz))) {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < Q; ++i) {   /* the rest direction is the site itself: solid */
                int X = x + C[i][0], Y = y + C[i][1], Z = z + C[i][2];
                if (is_solid(p, X, Y, Z)) continue;
                num += W[i] * rho_b[cell_index(p, wrap(X, p->nx), wrap(Y, p->ny), wrap(Z, p->nz))];
                den += W[i];
            }
            return (den > 0.0 ? num / den : 0.0) + rho_s;
        }
    }
    int mx = x, my = y, mz = z;
    if (!p->periodic[0]) { if (mx < 0) mx = -1 - mx; else if (mx >= p->nx) mx = 2 * p->nx - 1 - mx; }
    else mx = wrap(mx, p->nx);
    if (!p->periodic[1]) { if (my < 0) my = -1 - my; else if (my >= p->ny) my = 2 * p->ny - 1 - my; }
    else my = wrap(my, p->ny);
    if (!p->periodic[2]) { if (mz < 0) mz = -1 - mz; else if (mz >= p->nz) mz = 2 * p->nz - 1 - mz; }
    else mz = wrap(mz, p->nz);
    /* a mirror cell that is itself solid presents its own wall density */
    if (mask_solid(p, mx, my, mz)) return wall_density(p, rho_b, rho_s, mx, my, mz);
    return rho_b[cell_index(p, mx, my, mz)] + rho_s;
}

/* Interaction sums of Eq. 7 and Eq. 13 for one density field rho^b:
 *   S_fluid(x) = sum_{i: x+c_i fluid} w_i c_i rho^b(x + c_i)
 *   S_wall(x)  = sum_{i: x+c_i solid} w_i c_i rho'_b(x + c_i)
 * so that F^{ab} = G^{ab} rho^a S_fluid and F_w^{ab} = G^{ab} rho^a S_wall. */
void oracle_interaction_sums(const oracle_params *p, const double *rho_b, double rho_s_b,
                             double *S_fluid, double *S_wall)
{
    build_lattice();
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long s = cell_index(p, x, y, z);
                double sf[3] = {0, 0, 0}, sw[3] = {0, 0, 0};
                for (int i = 0; i < Q; ++i) {
                    int X = x + C[i][0], Y = y + C[i][1], Z = z + C[i][2];
                    double r;
                    if (is_solid(p, X, Y, Z)) {
                        r = wall_density(p, rho_b, rho_s_b, X, Y, Z);
                        for (int d = 0; d < 3; ++d) sw[d] += W[i] * C[i][d] * r;
                    } else {
                        r = rho_b[cell_index(p, wrap(X, p->nx), wrap(Y, p->ny), wrap(Z, p->nz))];
                        for (int d = 0; d < 3; ++d) sf[d] += W[i] * C[i][d] * r;
                    }
                }
                for (int d = 0; d < 3; ++d) {
                    S_fluid[3 * s + d] = sf[d];
                    S_wall[3 * s + d] = sw[d];
                }
            }
}

/* Acceleration of each component (text after Eq. 9):
 *   g^a = sum_b (F^{ab} + F_w^{ab}) / rho^a + g_ext,
 * with F^{ab} of Eq. 7 and F_w^{ab} of Eq. 13. */
void oracle_accelerations(const oracle_params *p, const double *rho1, const double *rho2,
                          double *g1, double *g2)
{
    long N = (long)p->nx * p->ny * p->nz;
    double *Sf[2], *Sw[2];
    const double *rho[2] = {rho1, rho2};
    double *g[2] = {g1, g2};
    for (int b = 0; b < 2; ++b) {
        Sf[b] = (double *)malloc(sizeof(double) * 3 * N);
        Sw[b] = (double *)malloc(sizeof(double) * 3 * N);
        oracle_interaction_sums(p, rho[b], p->rho_s[b], Sf[b], Sw[b]);
    }
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
    for (long s = 0; s < N; ++s)
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) {
                if (p->solid && p->solid[s]) { g[a][3 * s + d] = 0.0; continue; }
                double Fsum = 0.0;
                for (int b = 0; b < 2; ++b) {
                    double F = p->G[a][b] * rho[a][s] * Sf[b][3 * s + d];
                    double Fw = p->G[a][b] * rho[a][s] * Sw[b][3 * s + d];
                    Fsum += F + Fw;
                }
                g[a][3 * s + d] = Fsum / rho[a][s] + p->g_ext[d];
            }
    for (int b = 0; b < 2; ++b) { free(Sf[b]); free(Sw[b]); }
}

/* Collision of one component at one cell, producing the post-collision
 * populations fpost (the right-hand side of Eq. 1 or of Eq. 10).  u is the
 * velocity of the equilibrium: the mixture velocity of Eq. 6 for the
 * exact-difference forcing, the common u* = u + g/2 for Guo's forcing. */
static void collide_cell(const oracle_params *p, int a, const double fin[Q], double rho_a,
                         const double u[3], const double g_a[3], double fpost[Q])
{
    double feq[Q], Fi[Q];
    double tau = p->tau[a];
    oracle_feq(rho_a, u, feq);
    if (p->forcing == 1) {
        /* Guo, Zheng & Shi (2002): F_i = w_i [(c_i - u)/T0 + (c_i.u) c_i / T0^2] . F
         * with the component's force F = rho^a g^a */
        double F[3] = {rho_a * g_a[0], rho_a * g_a[1], rho_a * g_a[2]};
        for (int i = 0; i < Q; ++i) {
            double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += ((C[i][k] - u[k]) / T0 + cu * C[i][k] / (T0 * T0)) * F[k];
            Fi[i] = W[i] * s;
        }
        if (p->collision == 0) {
            /* Eq. 1 with the BGK operator of Eq. 2 and Guo's forcing */
            for (int i = 0; i < Q; ++i)
                fpost[i] = fin[i] - (fin[i] - feq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fi[i];
            return;
        }
        /* Eqs. 10-11 with Guo's forcing: the non-equilibrium part filtered is
         * f - f^eq + F/2, and F/2 is added after the collision */
        double d[Q];
        for (int i = 0; i < Q; ++i) d[i] = fin[i] - feq[i] + 0.5 * Fi[i];
        double Pi[3][3] = {{0}};
        for (int i = 0; i < Q; ++i)
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    Pi[r][c] += C[i][r] * C[i][c] * d[i];
        for (int i = 0; i < Q; ++i) {
            double contr = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    double Qrc = C[i][r] * C[i][c] - (r == c ? T0 : 0.0);
                    contr += Qrc * Pi[r][c];
                }
            double fneq = W[i] / (2.0 * T0 * T0) * contr;
            fpost[i] = feq[i] + (1.0 - 1.0 / tau) * fneq + 0.5 * Fi[i];
        }
        if (p->collision == 2) {
            for (int k = 0; k < N3; ++k) {
                double coef = 0.0;
                for (int i = 0; i < Q; ++i) coef += E3[k][i] * d[i];
                for (int i = 0; i < Q; ++i) fpost[i] += (1.0 - 1.0 / tau) * W[i] * E3[k][i] * coef;
            }
        }
        return;
    }
    {
        double ug[3] = {u[0] + g_a[0], u[1] + g_a[1], u[2] + g_a[2]};
        double feq_shift[Q];
        oracle_feq(rho_a, ug, feq_shift);
        /* forcing term: exact difference of equilibria (reading of Sec. 2) */
        for (int i = 0; i < Q; ++i) Fi[i] = feq_shift[i] - feq[i];
    }
    if (p->collision == 0) {
        /* Eq. 1 with the BGK operator of Eq. 2 */
        for (int i = 0; i < Q; ++i)
            fpost[i] = fin[i] - (fin[i] - feq[i]) / tau + Fi[i];
    } else {
        /* Eqs. 10-11: non-equilibrium momentum flux, then its Hermite projection */
        double Pi[3][3] = {{0}};
        for (int i = 0; i < Q; ++i)
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    Pi[r][c] += C[i][r] * C[i][c] * (fin[i] - feq[i]);
        for (int i = 0; i < Q; ++i) {
            double contr = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    double Qrc = C[i][r] * C[i][c] - (r == c ? T0 : 0.0);
                    contr += Qrc * Pi[r][c];
                }
            double fneq = W[i] / (2.0 * T0 * T0) * contr;
            fpost[i] = feq[i] + (1.0 - 1.0 / tau) * fneq + Fi[i];
        }
        if (p->collision == 2) {
            /* third-order part: w_i sum_k E3_k(c_i) <E3_k, (f - f^eq) / w> */
            for (int k = 0; k < N3; ++k) {
                double coef = 0.0;
                for (int i = 0; i < Q; ++i) coef += E3[k][i] * (fin[i] - feq[i]);
                for (int i = 0; i < Q; ++i) fpost[i] += (1.0 - 1.0 / tau) * W[i] * E3[k][i] * coef;
            }
        }
    }
}

/* Streaming, left-hand side of Eq. 1: f_i(x + c_i, t+1) = fpost_i(x, t),
 * periodic wrap, or half-way bounce-back where x + c_i is a wall site
 * (the population returns to x reversed). */
static void stream(const oracle_params *p, const double *fpost, double *fnew)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < Q; ++i)
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
            for (int z = 0; z < p->nz; ++z)
                for (int y = 0; y < p->ny; ++y)
                    for (int x = 0; x < p->nx; ++x) {
                        long s = cell_index(p, x, y, z);
                        if (p->solid && p->solid[s]) continue;   /* nothing leaves a solid site */
                        int X = x + C[i][0], Y = y + C[i][1], Z = z + C[i][2];
                        double v = fpost[((long)a * Q + i) * N + s];
                        if (is_solid(p, X, Y, Z))
                            fnew[((long)a * Q + OPP[i]) * N + s] = v;
                        else
                            fnew[((long)a * Q + i) * N +
                                 cell_index(p, wrap(X, p->nx), wrap(Y, p->ny), wrap(Z, p->nz))] = v;
                    }
}

/* One full time step in the paper's order; f is updated in place.
 * work must hold 2*19*N doubles. */
void oracle_step(const oracle_params *p, double *f, double *work, long nsteps)
{
    build_lattice();
    long N = (long)p->nx * p->ny * p->nz;
    double *rho1 = (double *)malloc(sizeof(double) * N);
    double *rho2 = (double *)malloc(sizeof(double) * N);
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    double *g1 = (double *)malloc(sizeof(double) * 3 * N);
    double *g2 = (double *)malloc(sizeof(double) * 3 * N);
    for (long t = 0; t < nsteps; ++t) {
        oracle_moments_raw(p, f, rho1, rho2, u);
        oracle_accelerations(p, rho1, rho2, g1, g2);
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
        for (long s = 0; s < N; ++s)
            for (int a = 0; a < 2; ++a) {
                double fin[Q], fpost[Q];
                if (p->solid && p->solid[s]) {   /* solid sites hold no populations */
                    for (int i = 0; i < Q; ++i) work[((long)a * Q + i) * N + s] = 0.0;
                    continue;
                }
                for (int i = 0; i < Q; ++i) fin[i] = f[((long)a * Q + i) * N + s];
                double ueq[3] = {u[3 * s], u[3 * s + 1], u[3 * s + 2]};
                if (p->forcing == 1)   /* common equilibrium velocity u + g/2 (Eqs. 8-9) */
                    for (int d = 0; d < 3; ++d)
                        ueq[d] += (rho1[s] * g1[3 * s + d] + rho2[s] * g2[3 * s + d]) / (2.0 * (rho1[s] + rho2[s]));
                collide_cell(p, a, fin, a == 0 ? rho1[s] : rho2[s], ueq,
                             a == 0 ? &g1[3 * s] : &g2[3 * s], fpost);
                for (int i = 0; i < Q; ++i) work[((long)a * Q + i) * N + s] = fpost[i];
            }
        stream(p, work, f);
    }
    free(rho1); free(rho2); free(u); free(g1); free(g2);
}

/* Initial state: f_i^a = f^eq_i(rho^a_0, u_0) (Eq. 3). u may be NULL (zero). */
void oracle_init(const oracle_params *p, const double *rho1, const double *rho2,
                 const double *u, double *f)
{
    build_lattice();
    long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
    for (long s = 0; s < N; ++s) {
        double uz[3] = {0, 0, 0};
        const double *us = u ? &u[3 * s] : uz;
        double feq[Q];
        for (int a = 0; a < 2; ++a) {
            oracle_feq(a == 0 ? rho1[s] : rho2[s], us, feq);
            for (int i = 0; i < Q; ++i) f[((long)a * Q + i) * N + s] = (p->solid && p->solid[s]) ? 0.0 : feq[i];
        }
    }
}

/* Output fields: rho^1, rho^2 and the velocity u_F = u + g/2 of Eqs. 8-9,
 * g = sum_a g^a rho^a / rho. */
void oracle_moments(const oracle_params *p, const double *f,
                    double *rho1, double *rho2, double *uF)
{
    long N = (long)p->nx * p->ny * p->nz;
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    double *g1 = (double *)malloc(sizeof(double) * 3 * N);
    double *g2 = (double *)malloc(sizeof(double) * 3 * N);
    oracle_moments_raw(p, f, rho1, rho2, u);
    oracle_accelerations(p, rho1, rho2, g1, g2);
#pragma omp parallel for schedule(static) if (OMP_BIG(p))
    for (long s = 0; s < N; ++s) {
        double rho = rho1[s] + rho2[s];
        if (p->solid && p->solid[s]) { uF[3 * s] = uF[3 * s + 1] = uF[3 * s + 2] = 0.0; continue; }
        for (int d = 0; d < 3; ++d) {
            double g = (g1[3 * s + d] * rho1[s] + g2[3 * s + d] * rho2[s]) / rho;
            uF[3 * s + d] = u[3 * s + d] + g / 2.0;
        }
    }
    free(u); free(g1); free(g2);
}

/* Post-collision populations of one cell and component, exposed so that
 * tests can check the collision alone (closed forms, invariants).  u is the
 * equilibrium velocity (with Guo's forcing the caller passes u + g/2). */
void oracle_collide_cell(const oracle_params *p, int a, const double fin[Q], double rho_a,
                         const double u[3], const double g_a[3], double fpost[Q])
{
    build_lattice();
    collide_cell(p, a, fin, rho_a, u, g_a, fpost);
}

/* Number of threads of the passes above (1 = plain serial loops); returns the
 * count in use, or 1 when the library was built without OpenMP. */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
