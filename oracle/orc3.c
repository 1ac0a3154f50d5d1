/*
 * orc3.c — FP64 CPU oracle of the same scheme in three dimensions, D3Q19.
 *
 * TEST INFRASTRUCTURE ONLY, like orc.c: the slow, literal statement of one
 * time step, loaded by the test suite and the benchmark's CPU legs only.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * The paper states the scheme on D2Q9 and says it carries over to other
 * lattices (Sec. 3, before Eq. 30).  This file takes D3Q19 (c_s^2 = 1/3):
 *   c_0 = 0 (w = 1/3); the 6 axis vectors (w = 1/18); the 12 edge
 *   diagonals (+-1, +-1, 0) and permutations (w = 1/36),
 * and applies every formula of Sec. 3 unchanged, with vectors of three
 * components: phi = sum g (Eq. 30), mu (Eq. 5), u (Eq. 31), p (Eq. 32),
 * f^eq, g^eq, F_i, G_i (Eqs. 24-29, Gamma_i = 1 + s_i), BGK collision
 * (Eqs. 22-23) and streaming.  The isotropic stencils take the same form
 * with the D3Q19 weights:
 *   grad chi(x) = (1/cs2) sum_{i>0} w_i c_i chi(x + c_i)
 *   lap  chi(x) = (2/cs2) sum_{i>0} w_i [chi(x + c_i) - chi(x)]
 * The body force is F_b = (0, -(rho - rho_ref) g, 0).  All three
 * directions are periodic.  kappa, beta, alpha and gamma are the 2-D
 * ones (they come from the 1-D interface profile and Eqs. 17, 33).
 *
 * Projected along z, D3Q19 gives exactly the D2Q9 weights (4/9, 1/9,
 * 1/36), and every formula above depends on the populations only through
 * moments and on c_i only through c_i . (u, F, grad): a field that does
 * not vary in z therefore evolves exactly as under the 2-D scheme.
 *
 * Build: compiled into liborc.so with orc.c (-ffp-contract=off).
 * Layout: pop[i * N + (z * ny + y) * nx + x], fields [(z * ny + y) * nx + x].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define ORC3_PAR _Pragma("omp parallel for schedule(static)")
#else
#define ORC3_PAR
#endif

#define Q 19
static const int CX3[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY3[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ3[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W3[Q] = {1.0 / 3.0,
                             1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2_3 = 1.0 / 3.0;
static const double PI_3D = 3.14159265358979323846;

/* Same field order as orc.c's parameter block (bc_x, bc_y must be 0). */
typedef struct {
    int nx, ny;
    double rho_A, rho_B, phi_A, phi_B;
    double sigma, W, M, tau_f, tau_g;
    double gravity, rho_ref;
    int bc_x, bc_y;
    double u_wall_bottom, u_wall_top;
} orc3_params;

typedef struct {
    orc3_params P;
    int nx, ny, nz;
    long N;
    double kappa, beta, lambda, alpha, gamma, drho, phibar;
    double *f, *g, *fs, *gs;
    double *phi, *rho, *mu, *lmu, *p;
    double *gph[3], *gmu[3], *F[3], *u[3], *gp[3];
    long step;
} orc3_sim;

static long id3(const orc3_sim *s, int x, int y, int z) {
    return ((long)z * s->ny + y) * s->nx + x;
}
static int wrap3(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
static double nb(const orc3_sim *s, const double *chi, int x, int y, int z) {
    return chi[id3(s, wrap3(x, s->nx), wrap3(y, s->ny), wrap3(z, s->nz))];
}

static void grad3(const orc3_sim *s, const double *chi, int x, int y, int z, double out[3]) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 1; i < Q; ++i) {
        double v = nb(s, chi, x + CX3[i], y + CY3[i], z + CZ3[i]);
        a += W3[i] * CX3[i] * v;
        b += W3[i] * CY3[i] * v;
        c += W3[i] * CZ3[i] * v;
    }
    out[0] = a / CS2_3;
    out[1] = b / CS2_3;
    out[2] = c / CS2_3;
}

static double lap3(const orc3_sim *s, const double *chi, int x, int y, int z) {
    double c0 = chi[id3(s, x, y, z)];
    double acc = 0.0;
    for (int i = 1; i < Q; ++i) acc += W3[i] * (nb(s, chi, x + CX3[i], y + CY3[i], z + CZ3[i]) - c0);
    return 2.0 * acc / CS2_3;
}

static double s3(int i, const double u[3]) {
    double cu = CX3[i] * u[0] + CY3[i] * u[1] + CZ3[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return cu / CS2_3 + (cu * cu - CS2_3 * uu) / (2.0 * CS2_3 * CS2_3);
}

static double mu_of(const orc3_sim *s, double ph, double lapphi) {
    return 4.0 * s->beta * (ph - s->P.phi_A) * (ph - s->P.phi_B) * (ph - s->phibar) - s->kappa * lapphi;
}

/* Passes 1-5 at the current time level. */
static void macro3(orc3_sim *s) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const long N = s->N;
    ORC3_PAR
    for (long k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int i = 0; i < Q; ++i) acc += s->g[i * N + k];
        s->phi[k] = acc;
        s->rho[k] = s->P.rho_B + (acc - s->P.phi_B) * s->drho;
    }
    ORC3_PAR
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = id3(s, x, y, z);
                s->mu[k] = mu_of(s, s->phi[k], lap3(s, s->phi, x, y, z));
            }
    ORC3_PAR
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = id3(s, x, y, z);
                double a[3], b[3];
                grad3(s, s->phi, x, y, z, a);
                grad3(s, s->mu, x, y, z, b);
                for (int d = 0; d < 3; ++d) {
                    s->gph[d][k] = a[d];
                    s->gmu[d][k] = b[d];
                }
                s->lmu[k] = lap3(s, s->mu, x, y, z);
            }
    ORC3_PAR
    for (long k = 0; k < N; ++k) {
        double ph = s->phi[k], rh = s->rho[k];
        double F[3] = {-ph * s->gmu[0][k], -ph * s->gmu[1][k] - (rh - s->P.rho_ref) * s->P.gravity,
                       -ph * s->gmu[2][k]};
        double sf = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[i * N + k];
            sf += fi;
            j[0] += CX3[i] * fi;
            j[1] += CY3[i] * fi;
            j[2] += CZ3[i] * fi;
        }
        double udr = 0.0;
        for (int d = 0; d < 3; ++d) {
            s->F[d][k] = F[d];
            s->u[d][k] = (j[d] + 0.5 * CS2_3 * F[d]) / (CS2_3 * rh);
            udr += s->u[d][k] * s->drho * s->gph[d][k];
        }
        s->p[k] = sf + 0.5 * CS2_3 * (udr - s->gamma * rh * s->lambda * s->lmu[k]);
    }
    ORC3_PAR
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = id3(s, x, y, z);
                double a[3];
                grad3(s, s->p, x, y, z, a);
                for (int d = 0; d < 3; ++d) s->gp[d][k] = a[d];
            }
}

/* Collision (Eqs. 22-29) and streaming, periodic. */
static void collide_stream3(orc3_sim *s) {
    const long N = s->N;
    const double tf = s->P.tau_f, tg = s->P.tau_g;
    ORC3_PAR
    for (long k = 0; k < N; ++k) {
        double u[3] = {s->u[0][k], s->u[1][k], s->u[2][k]};
        double F[3] = {s->F[0][k], s->F[1][k], s->F[2][k]};
        double gr[3], gpF[3];
        for (int d = 0; d < 3; ++d) {
            gr[d] = s->drho * s->gph[d][k];
            gpF[d] = s->gp[d][k] - F[d];
        }
        double ph = s->phi[k], rh = s->rho[k], amu = s->alpha * s->mu[k];
        for (int i = 0; i < Q; ++i) {
            double c[3] = {CX3[i], CY3[i], CZ3[i]};
            double si = s3(i, u);
            double Gam = 1.0 + si;
            double H = (i == 0) ? ph - (1.0 - W3[0]) * amu : W3[i] * amu;
            double feq = W3[i] * (s->p[k] + CS2_3 * rh * si);
            double geq = H + W3[i] * ph * si;
            double eF = 0.0, eR = 0.0, eD = 0.0;
            for (int d = 0; d < 3; ++d) {
                eF += (c[d] - u[d]) * F[d];
                eR += (c[d] - u[d]) * gr[d];
                eD += (c[d] - u[d]) * gpF[d];
            }
            double Fi = W3[i] * Gam * eF + W3[i] * si * CS2_3 * eR
                        - W3[i] * CS2_3 * rh * s->gamma * s->lambda * s->lmu[k];
            double Gi = -(ph / (CS2_3 * rh)) * W3[i] * Gam * eD;
            double fi = s->f[i * N + k], gi = s->g[i * N + k];
            s->fs[i * N + k] = fi - (fi - feq) / tf + (1.0 - 0.5 / tf) * Fi;
            s->gs[i * N + k] = gi - (gi - geq) / tg + (1.0 - 0.5 / tg) * Gi;
        }
    }
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    ORC3_PAR
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = id3(s, x, y, z);
                for (int i = 0; i < Q; ++i) {
                    long kd = id3(s, wrap3(x + CX3[i], nx), wrap3(y + CY3[i], ny), wrap3(z + CZ3[i], nz));
                    s->f[i * N + kd] = s->fs[i * N + k];
                    s->g[i * N + kd] = s->gs[i * N + k];
                }
            }
}

/* ------------------------------------------------------------ public API */

orc3_sim *orc3_create(const orc3_params *P, int nz) {
    if (!P || P->nx < 3 || P->ny < 3 || nz < 3) return NULL;
    if (!(P->tau_f > 0.5) || !(P->tau_g > 0.5) || !(P->rho_A > 0.0) || !(P->rho_B > 0.0)) return NULL;
    if (!(P->W > 0.0) || P->phi_A == P->phi_B || P->bc_x != 0 || P->bc_y != 0) return NULL;
    if (P->rho_B * P->phi_A - P->rho_A * P->phi_B == 0.0) return NULL;
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return NULL;
    s->P = *P;
    s->nx = P->nx;
    s->ny = P->ny;
    s->nz = nz;
    s->N = (long)P->nx * P->ny * nz;
    double d = P->phi_A - P->phi_B;
    s->phibar = 0.5 * (P->phi_A + P->phi_B);
    s->kappa = 3.0 * P->sigma * P->W / (2.0 * d * d);
    s->beta = 12.0 * P->sigma / (P->W * d * d * d * d);
    s->lambda = P->M;
    s->alpha = P->M / (CS2_3 * (P->tau_g - 0.5));
    s->drho = (P->rho_A - P->rho_B) / d;
    s->gamma = (P->rho_A - P->rho_B) / (P->rho_B * P->phi_A - P->rho_A * P->phi_B);
    const long N = s->N;
    double **pops[4] = {&s->f, &s->g, &s->fs, &s->gs};
    for (int b = 0; b < 4; ++b)
        if (!(*pops[b] = (double *)calloc((size_t)(Q * N), sizeof(double)))) return NULL;
    double **flds[20] = {&s->phi, &s->rho, &s->mu, &s->lmu, &s->p,
                         &s->gph[0], &s->gph[1], &s->gph[2], &s->gmu[0], &s->gmu[1], &s->gmu[2],
                         &s->F[0], &s->F[1], &s->F[2], &s->u[0], &s->u[1], &s->u[2],
                         &s->gp[0], &s->gp[1], &s->gp[2]};
    for (int b = 0; b < 20; ++b)
        if (!(*flds[b] = (double *)calloc((size_t)N, sizeof(double)))) return NULL;
    return s;
}

void orc3_destroy(orc3_sim *s) {
    if (!s) return;
    double *all[24] = {s->f, s->g, s->fs, s->gs, s->phi, s->rho, s->mu, s->lmu, s->p,
                       s->gph[0], s->gph[1], s->gph[2], s->gmu[0], s->gmu[1], s->gmu[2],
                       s->F[0], s->F[1], s->F[2], s->u[0], s->u[1], s->u[2],
                       s->gp[0], s->gp[1], s->gp[2]};
    for (int b = 0; b < 24; ++b) free(all[b]);
    free(s);
}

/* Equilibrium initial state: p = 0, u = u0 (0 where NULL), mu from phi0. */
void orc3_init_phi(orc3_sim *s, const double *phi0, const double *ux0, const double *uy0,
                   const double *uz0) {
    const long N = s->N;
    for (long k = 0; k < N; ++k) {
        s->phi[k] = phi0[k];
        s->rho[k] = s->P.rho_B + (phi0[k] - s->P.phi_B) * s->drho;
    }
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long k = id3(s, x, y, z);
                s->mu[k] = mu_of(s, s->phi[k], lap3(s, s->phi, x, y, z));
            }
    for (long k = 0; k < N; ++k) {
        double u[3] = {ux0 ? ux0[k] : 0.0, uy0 ? uy0[k] : 0.0, uz0 ? uz0[k] : 0.0};
        double amu = s->alpha * s->mu[k];
        for (int i = 0; i < Q; ++i) {
            double si = s3(i, u);
            double H = (i == 0) ? s->phi[k] - (1.0 - W3[0]) * amu : W3[i] * amu;
            s->f[i * N + k] = W3[i] * CS2_3 * s->rho[k] * si;
            s->g[i * N + k] = H + W3[i] * s->phi[k] * si;
        }
    }
    s->step = 0;
}

void orc3_step(orc3_sim *s, long n) {
    for (long t = 0; t < n; ++t) {
        macro3(s);
        collide_stream3(s);
        s->step++;
    }
}

/* Macroscopic fields of the current time level; any pointer may be NULL. */
void orc3_fields(orc3_sim *s, double *phi, double *rho, double *p, double *ux, double *uy,
                 double *uz, double *mu) {
    macro3(s);
    size_t b = (size_t)s->N * sizeof(double);
    if (phi) memcpy(phi, s->phi, b);
    if (rho) memcpy(rho, s->rho, b);
    if (p) memcpy(p, s->p, b);
    if (ux) memcpy(ux, s->u[0], b);
    if (uy) memcpy(uy, s->u[1], b);
    if (uz) memcpy(uz, s->u[2], b);
    if (mu) memcpy(mu, s->mu, b);
}

void orc3_mass(orc3_sim *s, double *mass, double *phi_total) {
    double m = 0.0, t = 0.0;
    for (long k = 0; k < s->N; ++k) {
        double ph = 0.0;
        for (int i = 0; i < Q; ++i) ph += s->g[i * s->N + k];
        t += ph;
        m += s->P.rho_B + (ph - s->P.phi_B) * s->drho;
    }
    *mass = m;
    *phi_total = t;
}

/* Laplace diagnostic of a droplet centred at (xc, yc, zc) with nominal
 * radius R: total pressure P = p0 - kappa phi lap phi + kappa |grad phi|^2/2 + p
 * (Sec. 4.2), p0 = phi psi' - psi; dP = mean over r < R - 2W minus mean over
 * r > R + 2W (nearest periodic image); R_eff from the volume of fluid A. */
void orc3_laplace(orc3_sim *s, double xc, double yc, double zc, double R, double *dP,
                  double *R_eff) {
    macro3(s);
    const double W = s->P.W, pa = s->P.phi_A, pb = s->P.phi_B;
    double sin_ = 0.0, sout = 0.0, vol = 0.0;
    long nin = 0, nout = 0;
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long k = id3(s, x, y, z);
                double ph = s->phi[k], g3[3];
                grad3(s, s->phi, x, y, z, g3);
                double psi = s->beta * (ph - pa) * (ph - pa) * (ph - pb) * (ph - pb);
                double dpsi = 4.0 * s->beta * (ph - pa) * (ph - pb) * (ph - s->phibar);
                double lp = lap3(s, s->phi, x, y, z);
                double gg = g3[0] * g3[0] + g3[1] * g3[1] + g3[2] * g3[2];
                double P = ph * dpsi - psi - s->kappa * ph * lp + 0.5 * s->kappa * gg + s->p[k];
                double dx = fabs(x - xc), dy = fabs(y - yc), dz = fabs(z - zc);
                dx = fmin(dx, s->nx - dx);
                dy = fmin(dy, s->ny - dy);
                dz = fmin(dz, s->nz - dz);
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (r < R - 2.0 * W) {
                    sin_ += P;
                    ++nin;
                } else if (r > R + 2.0 * W) {
                    sout += P;
                    ++nout;
                }
                vol += (ph - pb) / (pa - pb);
            }
    *dP = (nin ? sin_ / nin : 0.0) - (nout ? sout / nout : 0.0);
    *R_eff = cbrt(3.0 * vol / (4.0 * PI_3D));
}

void orc3_get_pops(const orc3_sim *s, double *f, double *g) {
    memcpy(f, s->f, (size_t)(Q * s->N) * sizeof(double));
    memcpy(g, s->g, (size_t)(Q * s->N) * sizeof(double));
}

long orc3_step_count(const orc3_sim *s) { return s->step; }

/* The isotropic gradient and Laplacian of a periodic field chi (for the
 * stencil tests). */
void orc3_stencils(int nx, int ny, int nz, const double *chi, double *gx, double *gy, double *gz,
                   double *lap) {
    orc3_sim s;
    memset(&s, 0, sizeof s);
    s.nx = nx;
    s.ny = ny;
    s.nz = nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = id3(&s, x, y, z);
                double a[3];
                grad3(&s, chi, x, y, z, a);
                gx[k] = a[0];
                gy[k] = a[1];
                gz[k] = a[2];
                lap[k] = lap3(&s, chi, x, y, z);
            }
}

void orc3_lattice(int *cx, int *cy, int *cz, double *w) {
    for (int i = 0; i < Q; ++i) {
        cx[i] = CX3[i];
        cy[i] = CY3[i];
        cz[i] = CZ3[i];
        w[i] = W3[i];
    }
}
