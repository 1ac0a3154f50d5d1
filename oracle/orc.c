/*
 * orc.c — FP64 CPU oracle of the quasi-incompressible phase-field lattice
 * Boltzmann scheme (Yang & Guo, arXiv 1507.03521), D2Q9.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal statement of what
 * one time step computes.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table
 * or constant with the CUDA library, and it never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared orc.c -o liborc.so -lm
 * (-ffp-contract=off: every product and sum is rounded separately, in the
 * order written, so results are reproducible across machines.)
 *
 * Naming follows the paper: f_i is the flow (hydrodynamic) population,
 * relaxed with tau_f (viscosity); g_i is the phase-field population, relaxed
 * with tau_g (mobility).  Sec. 3, below Eq. 23.
 *
 * One step (orc_step) is a sequence of full passes over the grid, each one a
 * formula of Sec. 3, in this order:
 *   1. phi = sum_i g_i (Eq. 30); rho from phi (Eq. 11)
 *   2. mu = psi'(phi) - kappa lap(phi) (Eq. 5)
 *   3. grad phi, grad rho = (drho/dphi) grad phi (Eq. 13), grad mu, lap mu
 *   4. F = -phi grad mu + F_b (Sec. 2 below Eq. 17; F_b of Sec. 4.3);
 *      u (Eq. 31); p (Eq. 32)
 *   5. grad p
 *   6. collision of f (Eq. 22) and g (Eq. 23) with f^eq (Eq. 24),
 *      g^eq (Eqs. 25-27), F_i (Eq. 28), G_i (Eq. 29)
 *   7. streaming (left-hand sides of Eqs. 22-23), with periodic wrap or
 *      halfway bounce-back at walls
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - Gamma_i(u), used in Eqs. 28-29 but never defined, is 1 + s_i(u): with it
 *    the zeroth and first moments printed in the appendix (Eqs. 52-53, 73)
 *    hold exactly.
 *  - "isotropic central scheme" (end of Sec. 3): for a field chi,
 *      grad chi(x) = (1/cs2) sum_{i=1..8} w_i c_i chi(x + c_i)
 *      lap  chi(x) = (2/cs2) sum_{i=1..8} w_i [chi(x + c_i) - chi(x)]
 *    and div(lambda grad mu) is lambda * lap(mu) (lambda constant).
 *  - grad p in G_i is taken at the same time level t as everything else.
 *  - Walls (not in the paper) sit on y = -1/2 and y = ny - 1/2: halfway
 *    bounce-back with a moving-wall term from the linear part of each
 *    equilibrium; stencil ghost rows mirror phi and mu (zero normal
 *    derivative) and extrapolate p linearly.
 *  - Body force F_b = (0, -(rho - rho_ref) g) (Sec. 4.3 uses rho_ref = rho_A).
 *  - Initial populations are the equilibria at p = 0 and the given u0, with
 *    mu from the initial phi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

/* ORC_MUTANT (default 0) plants one known mistake in the oracle so that the
 * test suite can show each of its pins catches one.  Only the mutation test
 * builds with a non-zero value; the oracle proper is built without it. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#include <string.h>
#include <stdio.h>

/* Built with -fopenmp (liborc_omp.so), the passes whose iterations write
 * disjoint cells run over all host cores; the arithmetic of every cell is
 * unchanged, so that build is bit-identical to the serial one.  Reductions
 * (mass, Laplace means) stay serial to keep their summation order. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_PAR_ROWS _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PAR_ROWS
#endif

/* D2Q9 velocities and weights, Sec. 3 (end): c_0 = 0, c_1..4 axis-aligned at
 * angles (i-1)pi/2, c_5..8 diagonal at angles (2i-1)pi/4. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;

enum { ORC_PERIODIC = 0, ORC_WALL = 1 };

typedef struct {
    int nx, ny;
    double rho_A, rho_B, phi_A, phi_B;
    double sigma, W, M, tau_f, tau_g;
    double gravity, rho_ref;
    int bc_x, bc_y;
    double u_wall_bottom, u_wall_top;
} orc_params;

typedef struct {
    orc_params P;
    long N;
    /* derived constants */
    double kappa, beta, lambda, alpha, gamma, drho, phibar, dphi, nu;
    /* populations at the current time, SoA: pop[i*N + y*nx + x] */
    double *f, *g;
    /* post-collision populations */
    double *fs, *gs;
    /* macroscopic fields of the current time level (passes 1-5) */
    double *phi, *rho, *mu, *gphx, *gphy, *grhx, *grhy, *gmux, *gmuy, *lmu;
    double *Fx, *Fy, *ux, *uy, *p, *gpx, *gpy;
    /* lagged variant: grad p in G_i from the previous step's p (pprev) */
    int lag;
    double *pprev;
    long step;
} orc_sim;

/* ---------------------------------------------------------------- helpers */

static long idx(const orc_sim *s, int x, int y) { return (long)y * s->P.nx + x; }

/* Periodic wrap along x (only periodic x is supported). */
static int wrapx(const orc_sim *s, int x) {
    int nx = s->P.nx;
    x %= nx;
    if (x < 0) x += nx;
    return x;
}

/* Row used for a stencil neighbour at row y: periodic wrap, or the even
 * mirror across a wall at y = -1/2 (row -1 -> 0, -2 -> 1, ...) and at
 * y = ny - 1/2 (row ny -> ny-1, ...). */
static int rowmap(const orc_sim *s, int y) {
    int ny = s->P.ny;
    if (s->P.bc_y == ORC_PERIODIC) {
        y %= ny;
        if (y < 0) y += ny;
        return y;
    }
    if (y < 0) return -y - 1;
    if (y >= ny) return 2 * ny - 1 - y;
    return y;
}

/* Field value of chi at (x, y) for phi-like fields (mirror at walls). */
static double at_mirror(const orc_sim *s, const double *chi, int x, int y) {
    return chi[idx(s, wrapx(s, x), rowmap(s, y))];
}

/* Field value of p at (x, y): periodic wrap, or linear extrapolation across
 * a wall, p(-1) = 2 p(0) - p(1) and p(ny) = 2 p(ny-1) - p(ny-2). */
static double at_extrap(const orc_sim *s, const double *chi, int x, int y) {
    int ny = s->P.ny;
    int xx = wrapx(s, x);
    if (s->P.bc_y == ORC_PERIODIC || (y >= 0 && y < ny))
        return chi[idx(s, xx, rowmap(s, y))];
    if (y < 0) return 2.0 * chi[idx(s, xx, 0)] - chi[idx(s, xx, 1)];
    return 2.0 * chi[idx(s, xx, ny - 1)] - chi[idx(s, xx, ny - 2)];
}

/* Isotropic central gradient (reading of the end of Sec. 3). */
static void grad_at(const orc_sim *s, const double *chi, int x, int y, int extrap,
                    double *gx, double *gy) {
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; ++i) {
        double v = extrap ? at_extrap(s, chi, x + CX[i], y + CY[i])
                          : at_mirror(s, chi, x + CX[i], y + CY[i]);
        sx += WT[i] * ((ORC_MUTANT == 6) ? CY[i] : CX[i]) * v;
        sy += WT[i] * ((ORC_MUTANT == 6) ? CX[i] : CY[i]) * v;
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}

/* Isotropic central Laplacian (reading of the end of Sec. 3). */
static double lap_at(const orc_sim *s, const double *chi, int x, int y) {
    double c = chi[idx(s, x, y)];
    double acc = 0.0;
    for (int i = 1; i < 9; ++i)
        acc += WT[i] * (at_mirror(s, chi, x + CX[i], y + CY[i]) - c);
    return 2.0 * acc / CS2;
}

/* s_i(u), Eq. 26. */
static double s_i(int i, double ux, double uy) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2);
}

/* ----------------------------------------------------- per-cell formulas */

/* f^eq (Eq. 24), g^eq (Eqs. 25, 27), F_i (Eq. 28) and G_i (Eq. 29) of one
 * cell, with Gamma_i = 1 + s_i. */
static void cell_terms(double alpha, double gamma, double lambda,
                       double phi, double mu, double p, double rho,
                       double ux, double uy, double Fx, double Fy,
                       double grhx, double grhy, double lmu,
                       double gpx, double gpy,
                       double *feq, double *geq, double *Fi, double *Gi) {
    for (int i = 0; i < 9; ++i) {
        double si = s_i(i, ux, uy);
        double Gam = (ORC_MUTANT == 1) ? 1.0 : 1.0 + si;
        double H = (i == 0) ? phi - ((ORC_MUTANT == 5) ? WT[0] : (1.0 - WT[0])) * alpha * mu
                            : WT[i] * alpha * mu;
        const double sgr = (ORC_MUTANT == 2) ? -1.0 : 1.0;
        const double irho = (ORC_MUTANT == 9) ? 1.0 : 1.0 / rho;
        feq[i] = WT[i] * (p + CS2 * rho * si);
        geq[i] = H + WT[i] * phi * si;
        double ex = CX[i] - ux, ey = CY[i] - uy;
        Fi[i] = ex * (WT[i] * Gam * Fx + sgr * WT[i] * si * CS2 * grhx)
              + ey * (WT[i] * Gam * Fy + sgr * WT[i] * si * CS2 * grhy)
              - ((ORC_MUTANT == 7) ? -1.0 : 1.0) * WT[i] * CS2 * rho * gamma * lambda * lmu;
        Gi[i] = -(phi * irho / CS2) * (ex * (gpx - Fx) + ey * (gpy - Fy)) * WT[i] * Gam;
    }
}

/* ------------------------------------------------------------- the passes */

/* Passes 1-5: macroscopic fields at the current time level. */
static void macroscopic(orc_sim *s) {
    const int nx = s->P.nx, ny = s->P.ny;
    const long N = s->N;
    /* pass 1: phi (Eq. 30), rho (Eq. 11) */
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double acc = 0.0;
            for (int i = 0; i < 9; ++i) acc += s->g[i * N + k];
            s->phi[k] = acc;
            s->rho[k] = s->P.rho_B + (acc - s->P.phi_B) * s->drho;
        }
    /* pass 2: chemical potential (Eq. 5) */
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double ph = s->phi[k];
            double dpsi = 4.0 * s->beta * (ph - s->P.phi_A) * (ph - s->P.phi_B) * (ph - s->phibar);
            s->mu[k] = dpsi - ((ORC_MUTANT == 11) ? -1.0 : 1.0) * s->kappa * lap_at(s, s->phi, x, y);
        }
    /* pass 3: gradients */
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            grad_at(s, s->phi, x, y, 0, &s->gphx[k], &s->gphy[k]);
            s->grhx[k] = s->drho * s->gphx[k];
            s->grhy[k] = s->drho * s->gphy[k];
            grad_at(s, s->mu, x, y, 0, &s->gmux[k], &s->gmuy[k]);
            s->lmu[k] = lap_at(s, s->mu, x, y);
        }
    /* pass 4: force, velocity (Eq. 31), pressure (Eq. 32) */
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double ph = s->phi[k], rh = s->rho[k];
            double Fx = -ph * s->gmux[k];
            double Fy = -ph * s->gmuy[k] - (rh - s->P.rho_ref) * s->P.gravity;
            double sf = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                double fi = s->f[i * N + k];
                sf += fi;
                jx += CX[i] * fi;
                jy += CY[i] * fi;
            }
            const double hf = (ORC_MUTANT == 3) ? 0.0 : 0.5;
            double ux = (jx + hf * CS2 * Fx) / (CS2 * rh);
            double uy = (jy + hf * CS2 * Fy) / (CS2 * rh);
            double udr = ux * s->grhx[k] + uy * s->grhy[k];
            s->Fx[k] = Fx;
            s->Fy[k] = Fy;
            s->ux[k] = ux;
            s->uy[k] = uy;
            s->p[k] = sf + 0.5 * CS2 * (udr - ((ORC_MUTANT == 8) ? 0.0 : 1.0) * s->gamma * rh * s->lambda * s->lmu[k]);
        }
    /* pass 5: pressure gradient (of the previous step's p in the lagged
     * variant) */
    const double *pg = s->lag ? s->pprev : s->p;
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            grad_at(s, pg, x, y, 1, &s->gpx[k], &s->gpy[k]);
        }
}

/* Pass 6: collision of Eqs. 22-23. */
static void collide(orc_sim *s) {
    const long N = s->N;
    const double tf = s->P.tau_f, tg = s->P.tau_g;
    ORC_PAR_ROWS
    for (long k = 0; k < N; ++k) {
        double feq[9], geq[9], Fi[9], Gi[9];
        cell_terms(s->alpha, s->gamma, s->lambda, s->phi[k], s->mu[k], s->p[k], s->rho[k],
                   s->ux[k], s->uy[k], s->Fx[k], s->Fy[k], s->grhx[k], s->grhy[k],
                   s->lmu[k], s->gpx[k], s->gpy[k], feq, geq, Fi, Gi);
        for (int i = 0; i < 9; ++i) {
            double fi = s->f[i * N + k], gi = s->g[i * N + k];
            const double pf = (ORC_MUTANT == 4) ? 1.0 : (1.0 - 1.0 / (2.0 * tf));
            const double pg = (ORC_MUTANT == 4) ? 1.0 : (1.0 - 1.0 / (2.0 * tg));
            s->fs[i * N + k] = fi - (fi - feq[i]) / tf + pf * Fi[i];
            s->gs[i * N + k] = gi - (gi - geq[i]) / tg + pg * Gi[i];
        }
    }
}

/* Pass 7: streaming, f_i(x + c_i, t + 1) = f_i*(x, t), with halfway
 * bounce-back at y walls: a population leaving the domain returns to its
 * own node in the opposite direction, minus twice the linear term of its
 * equilibrium evaluated at the wall velocity (u_w, 0). */
static void stream(orc_sim *s) {
    const int nx = s->P.nx, ny = s->P.ny;
    const long N = s->N;
    ORC_PAR_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            for (int i = 0; i < 9; ++i) {
                int yd = y + CY[i];
                int out = (s->P.bc_y == ORC_WALL) && (yd < 0 || yd >= ny);
                if (out) {
                    double uw = (yd < 0) ? s->P.u_wall_bottom : s->P.u_wall_top;
                    double cu = (ORC_MUTANT == 10) ? 0.0 : CX[i] * uw;
                    int o = OPP[i];
                    s->f[o * N + k] = s->fs[i * N + k] - 2.0 * WT[i] * s->rho[k] * cu;
                    s->g[o * N + k] = s->gs[i * N + k] - 2.0 * WT[i] * s->phi[k] * cu / CS2;
                } else {
                    int xd = wrapx(s, x + CX[i]);
                    int yy = rowmap(s, yd);
                    long kd = idx(s, xd, yy);
                    s->f[i * N + kd] = s->fs[i * N + k];
                    s->g[i * N + kd] = s->gs[i * N + k];
                }
            }
        }
}

/* ------------------------------------------------------------- public API */

int orc_params_check(const orc_params *P) {
    if (!P) return -1;
    if (P->nx < 5 || P->ny < 5) return -1;
    if (!(P->tau_f > 0.5) || !(P->tau_g > 0.5)) return -1;
    if (!(P->rho_A > 0.0) || !(P->rho_B > 0.0)) return -1;
    if (!(P->W > 0.0) || !(P->sigma >= 0.0) || !(P->M >= 0.0)) return -1;
    if (P->phi_A == P->phi_B) return -1;
    if (P->bc_x != ORC_PERIODIC) return -1;
    if (P->bc_y != ORC_PERIODIC && P->bc_y != ORC_WALL) return -1;
    if (P->rho_B * P->phi_A - P->rho_A * P->phi_B == 0.0) return -1;
    return 0;
}

/* Derived constants (Eqs. 3, 4, 13, 17, 33). */
static void derive(orc_sim *s) {
    const orc_params *P = &s->P;
    double d = P->phi_A - P->phi_B;
    s->dphi = d;
    s->phibar = 0.5 * (P->phi_A + P->phi_B);
    /* Eqs. 3-4 solved for kappa and beta. */
    s->kappa = ((ORC_MUTANT == 12) ? 2.0 : 1.0) * 3.0 * P->sigma * P->W / (2.0 * d * d);
    s->beta = 12.0 * P->sigma / (P->W * d * d * d * d);
    s->lambda = P->M;
    s->alpha = P->M / (CS2 * (P->tau_g - 0.5)); /* Eq. 33 */
    s->nu = CS2 * (P->tau_f - 0.5);              /* Eq. 33 */
    s->drho = (P->rho_A - P->rho_B) / d;         /* Eq. 13 */
    /* Eq. 17: gamma = (rho_r - 1) / (phi_A - phi_B rho_r), rho_r = rho_A/rho_B */
    s->gamma = (P->rho_A - P->rho_B) / (P->rho_B * P->phi_A - P->rho_A * P->phi_B);
}

orc_sim *orc_create(const orc_params *P) {
    if (orc_params_check(P) != 0) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->P = *P;
    s->N = (long)P->nx * P->ny;
    derive(s);
    long N = s->N;
    double **bufs9[4] = {&s->f, &s->g, &s->fs, &s->gs};
    for (int b = 0; b < 4; ++b) {
        *bufs9[b] = (double *)calloc((size_t)(9 * N), sizeof(double));
        if (!*bufs9[b]) return NULL;
    }
    double **flds[18] = {&s->phi, &s->rho, &s->mu, &s->gphx, &s->gphy, &s->grhx, &s->grhy,
                         &s->gmux, &s->gmuy, &s->lmu, &s->Fx, &s->Fy, &s->ux, &s->uy,
                         &s->p, &s->gpx, &s->gpy, &s->pprev};
    for (int b = 0; b < 18; ++b) {
        *flds[b] = (double *)calloc((size_t)N, sizeof(double));
        if (!*flds[b]) return NULL;
    }
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    double *all[22] = {s->f, s->g, s->fs, s->gs, s->phi, s->rho, s->mu, s->gphx, s->gphy,
                       s->grhx, s->grhy, s->gmux, s->gmuy, s->lmu, s->Fx, s->Fy, s->ux,
                       s->uy, s->p, s->gpx, s->gpy, s->pprev};
    for (int b = 0; b < 22; ++b) free(all[b]);
    free(s);
}

/* Derived constants: kappa, beta, lambda, alpha, gamma, drho/dphi, nu. */
void orc_constants(const orc_sim *s, double *out7) {
    out7[0] = s->kappa;
    out7[1] = s->beta;
    out7[2] = s->lambda;
    out7[3] = s->alpha;
    out7[4] = s->gamma;
    out7[5] = s->drho;
    out7[6] = s->nu;
}

/* Equilibrium initial state: p = 0, u = u0 (zero where NULL), mu from phi0,
 * f = f^eq(0, rho0, u0), g = g^eq(phi0, mu0, u0). */
int orc_init_phi(orc_sim *s, const double *phi0, const double *ux0, const double *uy0) {
    const int nx = s->P.nx, ny = s->P.ny;
    const long N = s->N;
    for (long k = 0; k < N; ++k) {
        s->phi[k] = phi0[k];
        s->rho[k] = s->P.rho_B + (phi0[k] - s->P.phi_B) * s->drho;
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double ph = s->phi[k];
            double dpsi = 4.0 * s->beta * (ph - s->P.phi_A) * (ph - s->P.phi_B) * (ph - s->phibar);
            s->mu[k] = dpsi - s->kappa * lap_at(s, s->phi, x, y);
        }
    for (long k = 0; k < N; ++k) {
        double ux = ux0 ? ux0[k] : 0.0, uy = uy0 ? uy0[k] : 0.0;
        for (int i = 0; i < 9; ++i) {
            double si = s_i(i, ux, uy);
            double H = (i == 0) ? s->phi[k] - (1.0 - WT[0]) * s->alpha * s->mu[k]
                                : WT[i] * s->alpha * s->mu[k];
            s->f[i * N + k] = WT[i] * (0.0 + CS2 * s->rho[k] * si);
            s->g[i * N + k] = H + WT[i] * s->phi[k] * si;
        }
    }
    memset(s->pprev, 0, (size_t)N * sizeof(double));  /* the initial state's p */
    s->step = 0;
    return 0;
}

void orc_step(orc_sim *s, long n) {
    for (long t = 0; t < n; ++t) {
        macroscopic(s);
        collide(s);
        stream(s);
        if (s->lag) memcpy(s->pprev, s->p, (size_t)s->N * sizeof(double));
        s->step++;
    }
}

/* Conditioning probe for the tests; not part of the scheme.  Before each of
 * n steps every population moves by one unit in the last place, up or down
 * as the low bit of a counter-based hash of (seed, step, index) says (the
 * SplitMix64 finaliser of Steele, Lea and Flood, 2014).  How far the fields
 * then drift from an unperturbed run measures how strongly the run
 * amplifies roundoff injected at every step, which is what a second
 * implementation with another rounding order does to it. */
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

void orc_step_jitter(orc_sim *s, long n, unsigned long long seed) {
    const long N9 = 9 * s->N;
    for (long t = 0; t < n; ++t) {
        const uint64_t base = splitmix64((uint64_t)seed ^ ((uint64_t)s->step << 32));
        double *pop[2] = {s->f, s->g};
        for (int b = 0; b < 2; ++b) {
            double *a = pop[b];
            const uint64_t off = base + (uint64_t)b * (uint64_t)N9;
            ORC_PAR_ROWS
            for (long q = 0; q < N9; ++q)
                a[q] = nextafter(a[q], (splitmix64(off + (uint64_t)q) & 1) ? INFINITY : -INFINITY);
        }
        orc_step(s, 1);
    }
}

/* The lagged-grad-p variant (not in the paper; a measurement of what
 * synchrony costs): G_i of Eq. 29 takes grad p from the pressure of the
 * previous step instead of the current one, which makes the step reach 2
 * cells instead of 3.  Before the first step that pressure is the initial
 * state's, p = 0.  Set before orc_init_phi. */
void orc_set_gradp_lag(orc_sim *s, int on) { s->lag = on ? 1 : 0; }

/* Macroscopic fields of the current time level; any pointer may be NULL. */
void orc_fields(orc_sim *s, double *phi, double *rho, double *p, double *ux, double *uy,
                double *mu) {
    macroscopic(s);
    size_t b = (size_t)s->N * sizeof(double);
    if (phi) memcpy(phi, s->phi, b);
    if (rho) memcpy(rho, s->rho, b);
    if (p) memcpy(p, s->p, b);
    if (ux) memcpy(ux, s->ux, b);
    if (uy) memcpy(uy, s->uy, b);
    if (mu) memcpy(mu, s->mu, b);
}

/* Total mass sum rho and total order parameter sum phi, in cell order. */
void orc_mass(orc_sim *s, double *mass, double *phi_total) {
    double m = 0.0, t = 0.0;
    for (long k = 0; k < s->N; ++k) {
        double ph = 0.0;
        for (int i = 0; i < 9; ++i) ph += s->g[i * s->N + k];
        t += ph;
        m += s->P.rho_B + (ph - s->P.phi_B) * s->drho;
    }
    *mass = m;
    *phi_total = t;
}

/* Total pressure of Sec. 4.2, P = p0 - kappa phi lap(phi) + kappa |grad phi|^2/2 + p
 * with p0 = phi psi'(phi) - psi(phi). */
void orc_total_pressure(orc_sim *s, double *P) {
    macroscopic(s);
    const int nx = s->P.nx, ny = s->P.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double ph = s->phi[k];
            double a = ph - s->P.phi_A, b = ph - s->P.phi_B;
            double psi = s->beta * a * a * b * b;
            double dpsi = 4.0 * s->beta * a * b * (ph - s->phibar);
            double p0 = ph * dpsi - psi;
            double lph = lap_at(s, s->phi, x, y);
            double g2 = s->gphx[k] * s->gphx[k] + s->gphy[k] * s->gphy[k];
            P[k] = p0 - s->kappa * ph * lph + 0.5 * s->kappa * g2 + s->p[k];
        }
}

/* Laplace diagnostic of Sec. 4.2 for a droplet centred at (xc, yc) of
 * nominal radius R: dP = mean P over r < R - 2W minus mean P over r > R + 2W
 * (r measured with the nearest periodic image); R_eff = sqrt(A/pi) with
 * A = sum (phi - phi_B)/(phi_A - phi_B). */
void orc_laplace(orc_sim *s, double xc, double yc, double R, double *dP, double *R_eff) {
    const int nx = s->P.nx, ny = s->P.ny;
    double *P = (double *)malloc((size_t)s->N * sizeof(double));
    orc_total_pressure(s, P);
    double si = 0.0, so = 0.0, A = 0.0;
    long ni = 0, no = 0;
    double W = s->P.W;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(s, x, y);
            double dx = fabs(x - xc), dy = fabs(y - yc);
            if (dx > 0.5 * nx) dx = nx - dx;
            if (dy > 0.5 * ny) dy = ny - dy;
            double r = sqrt(dx * dx + dy * dy);
            if (r < R - 2.0 * W) { si += P[k]; ni++; }
            if (r > R + 2.0 * W) { so += P[k]; no++; }
            A += (s->phi[k] - s->P.phi_B) / s->dphi;
        }
    *dP = (ni > 0 && no > 0) ? si / ni - so / no : NAN;
    *R_eff = sqrt(A / 3.14159265358979323846);
    free(P);
}

/* Population state access (9*N doubles each, SoA). */
void orc_get_pops(const orc_sim *s, double *f, double *g) {
    size_t b = (size_t)(9 * s->N) * sizeof(double);
    if (f) memcpy(f, s->f, b);
    if (g) memcpy(g, s->g, b);
}

void orc_set_pops(orc_sim *s, const double *f, const double *g) {
    size_t b = (size_t)(9 * s->N) * sizeof(double);
    if (f) memcpy(s->f, f, b);
    if (g) memcpy(s->g, g, b);
}

long orc_step_count(const orc_sim *s) { return s->step; }

/* Threads of the OpenMP build (no effect in the serial build); returns the
 * number the passes will use. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Unit-test access to the per-cell formulas (Eqs. 24-29). */
void orc_cell_terms(double alpha, double gamma, double lambda,
                    double phi, double mu, double p, double rho,
                    double ux, double uy, double Fx, double Fy,
                    double grhx, double grhy, double lmu, double gpx, double gpy,
                    double *feq, double *geq, double *Fi, double *Gi) {
    cell_terms(alpha, gamma, lambda, phi, mu, p, rho, ux, uy, Fx, Fy, grhx, grhy, lmu, gpx,
               gpy, feq, geq, Fi, Gi);
}

/* Unit-test access to the stencils on an nx*ny field with the given y
 * boundary (0 periodic, 1 wall-mirror); extrap selects the p ghost rule. */
int orc_stencils(int nx, int ny, int bc_y, int extrap, const double *chi, double *gx,
                 double *gy, double *lap) {
    orc_sim s;
    memset(&s, 0, sizeof(s));
    s.P.nx = nx;
    s.P.ny = ny;
    s.P.bc_y = bc_y;
    s.N = (long)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = idx(&s, x, y);
            grad_at(&s, chi, x, y, extrap, &gx[k], &gy[k]);
            lap[k] = lap_at(&s, chi, x, y);
        }
    return 0;
}

/* D2Q9 tables for cross-checks in tests. */
void orc_lattice(int *cx, int *cy, double *w) {
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = WT[i];
    }
}
