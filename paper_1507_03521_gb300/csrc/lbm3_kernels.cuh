// lbm3_kernels.cuh — the step on D3Q19 (three dimensions, periodic).
//
// Every formula of Sec. 3 carries over with three-component vectors:
// phi = sum g (Eq. 30), mu (Eq. 5), u (Eq. 31), p (Eq. 32), the equilibria
// and sources of Eqs. 24-29 with Gamma_i = 1 + s_i, BGK (Eqs. 22-23) and
// streaming; the isotropic stencils use the D3Q19 weights:
//   grad chi = (1/cs2) sum_{i>0} w_i c_i chi(x + c_i)
//   lap  chi = (2/cs2) sum_{i>0} w_i [chi(x + c_i) - chi(x)]
// The body force is F_b = (0, -(rho - rho_ref) g, 0).
//
// One step is four passes over the grid (one thread per cell):
//   k3_phi      phi = sum g                                   -> phi field
//   k3_mu       mu from phi and its Laplacian                 -> mu field
//   k3_p        moments of f, grad phi, grad mu, lap mu, u, p -> p field
//   k3_collide  the same per-cell terms again, grad p, the collision and
//               the push into the other ping-pong level.
// The radius-3 coupling (grad p <- p <- lap mu <- lap phi) is carried by
// the three stored fields; stencil neighbours are read through the
// read-only cache.  Level layout: slots f_0..f_18, g_0..g_18 of NS
// elements, cell k = (z ny + y) nx + x.
#pragma once

#include <cuda_runtime.h>

namespace lbm3 {

struct D3Q19 {
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
               : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
               : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
               : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};
static_assert(D3Q19::cx(7) == 1 && D3Q19::cy(7) == 1 && D3Q19::cz(7) == 0, "edge (1,1,0)");
static_assert(D3Q19::cx(13) == 1 && D3Q19::cz(13) == -1, "edge (1,0,-1)");
static_assert(D3Q19::cy(18) == -1 && D3Q19::cz(18) == 1, "edge (0,-1,1)");

// Kernel parameters in the compute type T.
template <class T>
struct K3 {
    int nx, ny, nz;
    long long N, NS;
    T phiA, phiB, phibar, rhoB, drho;
    T kappa, beta4, alpha, gl, grav, rhoref;
    T itf, itg, pf, pg;
};

// Neighbour cells of a cell (periodic in x, y, z); grids stay below 2^31
// cells, so 32-bit indices.
struct Nbr3 {
    int k;
    int o[19];
    __device__ __forceinline__ Nbr3(int kk, int nx, int ny, int nz) : k(kk) {
        const int x = kk % nx;
        const int r = kk / nx;
        const int y = r % ny;
        const int z = r / ny;
        const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
        const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
#pragma unroll
        for (int i = 0; i < 19; ++i)
            o[i] = (zs[1 + D3Q19::cz(i)] * ny + ys[1 + D3Q19::cy(i)]) * nx + xs[1 + D3Q19::cx(i)];
    }
};

template <class T>
__device__ __forceinline__ void grad3(const T *__restrict__ a, const Nbr3 &n, T g[3]) {
    T sx = 0, sy = 0, sz = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const T v = T(D3Q19::w(i) * 3.0) * __ldg(a + n.o[i]);
        if (D3Q19::cx(i)) sx += D3Q19::cx(i) > 0 ? v : -v;
        if (D3Q19::cy(i)) sy += D3Q19::cy(i) > 0 ? v : -v;
        if (D3Q19::cz(i)) sz += D3Q19::cz(i) > 0 ? v : -v;
    }
    g[0] = sx;
    g[1] = sy;
    g[2] = sz;
}

template <class T>
__device__ __forceinline__ T lap3(const T *__restrict__ a, const Nbr3 &n) {
    const T c = __ldg(a + n.k);
    T ax = 0, ed = 0;  // axis and edge neighbours, differences first
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const T d = __ldg(a + n.o[i]) - c;
        if (i < 7) ax += d;
        else ed += d;
    }
    return T(2.0 * 3.0 / 18.0) * ax + T(2.0 * 3.0 / 36.0) * ed;
}

template <class T>
__device__ __forceinline__ T mu_of(const K3<T> &P, T ph, T lapphi) {
    return P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) - P.kappa * lapphi;
}

// Per-cell terms of passes 3 and 4: u (Eq. 31), F, lap mu, grad phi and
// p (Eq. 32) from the cell's f and the phi, mu fields.
template <class T>
struct Macro3 {
    T phi, rho, u[3], F[3], lm, gph[3], p;
};

template <class T>
__device__ __forceinline__ Macro3<T> macro3(const K3<T> &P, const T f[19], const T *__restrict__ phi,
                                            const T *__restrict__ mu, const Nbr3 &n) {
    Macro3<T> m;
    T sf = 0, j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        sf += f[i];
        if (D3Q19::cx(i)) j[0] += D3Q19::cx(i) > 0 ? f[i] : -f[i];
        if (D3Q19::cy(i)) j[1] += D3Q19::cy(i) > 0 ? f[i] : -f[i];
        if (D3Q19::cz(i)) j[2] += D3Q19::cz(i) > 0 ? f[i] : -f[i];
    }
    m.phi = __ldg(phi + n.k);
    m.rho = P.rhoB + (m.phi - P.phiB) * P.drho;
    T gm[3];
    grad3(phi, n, m.gph);
    grad3(mu, n, gm);
    m.lm = lap3(mu, n);
    m.F[0] = -m.phi * gm[0];
    m.F[1] = -m.phi * gm[1] - (m.rho - P.rhoref) * P.grav;
    m.F[2] = -m.phi * gm[2];
    const T irc = T(3) / m.rho;
    T udr = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        m.u[d] = (j[d] + T(0.5 / 3.0) * m.F[d]) * irc;
        udr += m.u[d] * m.gph[d];
    }
    m.p = sf + T(0.5 / 3.0) * (udr * P.drho - P.gl * m.rho * m.lm);
    return m;
}

template <class T>
__global__ void k3_phi(const T *__restrict__ lvl, T *__restrict__ phi, const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const T *g = lvl + 19 * P.NS + k;
    T s = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) s += __ldg(g + i * P.NS);
    phi[k] = s;
}

template <class T>
__global__ void k3_mu(const T *__restrict__ phi, T *__restrict__ mu, const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const Nbr3 n((int)k, P.nx, P.ny, P.nz);
    mu[k] = mu_of(P, __ldg(phi + k), lap3(phi, n));
}

template <class T>
__global__ void k3_p(const T *__restrict__ lvl, const T *__restrict__ phi, const T *__restrict__ mu,
                     T *__restrict__ p, const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const Nbr3 n((int)k, P.nx, P.ny, P.nz);
    T f[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = __ldg(lvl + i * P.NS + k);
    p[k] = macro3(P, f, phi, mu, n).p;
}

// Pass 4: collision (Eqs. 22-29, Gamma_i = 1 + s_i) and push.  FP32 is
// held to 128 registers (two 256-thread CTAs per SM; left free it took
// 144 and ran 20% slower).
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k3_collide(const T *__restrict__ src, T *__restrict__ dst, const T *__restrict__ phi,
                           const T *__restrict__ mu, const T *__restrict__ pf_, const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const Nbr3 n((int)k, P.nx, P.ny, P.nz);
    T f[19], g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        f[i] = __ldg(src + i * P.NS + k);
        g[i] = __ldg(src + (19 + i) * P.NS + k);
    }
    const Macro3<T> m = macro3(P, f, phi, mu, n);
    T gp[3];
    grad3(pf_, n, gp);
    const T ux = m.u[0], uy = m.u[1], uz = m.u[2];
    const T gr[3] = {P.drho * m.gph[0], P.drho * m.gph[1], P.drho * m.gph[2]};
    const T D[3] = {gp[0] - m.F[0], gp[1] - m.F[1], gp[2] - m.F[2]};
    const T uu15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
    const T uF = ux * m.F[0] + uy * m.F[1] + uz * m.F[2];
    const T uR = ux * gr[0] + uy * gr[1] + uz * gr[2];
    const T uD = ux * D[0] + uy * D[1] + uz * D[2];
    const T Q = P.pg * (T(-3) * m.phi / m.rho);           // pg * (-phi / (cs2 rho))
    const T Kf = P.itf * m.p - P.pf * (T(1.0 / 3.0) * m.rho * P.gl * m.lm);
    const T Bf = P.itf * (T(1.0 / 3.0) * m.rho);
    const T omf = T(1) - P.itf, omg = T(1) - P.itg;
    const T phg = P.itg * m.phi;
    const T Ag = P.itg * P.alpha * __ldg(mu + k);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T cx = T(D3Q19::cx(i)), cy = T(D3Q19::cy(i)), cz = T(D3Q19::cz(i));
        const T w = T(D3Q19::w(i));
        const T cu = cx * ux + cy * uy + cz * uz;
        const T si = cu * (T(3) + T(4.5) * cu) - uu15;        // s_i (Eq. 26)
        const T eF = (cx * m.F[0] + cy * m.F[1] + cz * m.F[2]) - uF;
        const T eR = T(1.0 / 3.0) * ((cx * gr[0] + cy * gr[1] + cz * gr[2]) - uR);
        const T eD = (cx * D[0] + cy * D[1] + cz * D[2]) - uD;
        const T fv = omf * f[i] + w * (Kf + Bf * si + P.pf * (eF + si * (eF + eR)));
        const T Hg = (i == 0) ? (phg - T(1.0 - D3Q19::w(0)) * Ag) * T(1.0 / D3Q19::w(0)) : Ag;
        const T gv = omg * g[i] + w * (Hg + phg * si + Q * (eD + si * eD));
        const long long kd = n.o[i];
        dst[i * P.NS + kd] = fv;
        dst[(19 + i) * P.NS + kd] = gv;
    }
}

// Equilibrium initial state (p = 0, u = u0, mu from phi0): f = f^eq,
// g = g^eq.  mu must hold mu(phi0) (k3_mu on phi0).
template <class T>
__global__ void k3_init(const T *__restrict__ phi0, const T *__restrict__ mu,
                        const T *__restrict__ ux0, const T *__restrict__ uy0,
                        const T *__restrict__ uz0, T *__restrict__ lvl, const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const T ph = phi0[k];
    const T rho = P.rhoB + (ph - P.phiB) * P.drho;
    const T u[3] = {ux0 ? ux0[k] : T(0), uy0 ? uy0[k] : T(0), uz0 ? uz0[k] : T(0)};
    const T uu15 = T(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const T amu = P.alpha * mu[k];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T cu = T(D3Q19::cx(i)) * u[0] + T(D3Q19::cy(i)) * u[1] + T(D3Q19::cz(i)) * u[2];
        const T si = cu * (T(3) + T(4.5) * cu) - uu15;
        const T w = T(D3Q19::w(i));
        const T H = (i == 0) ? ph - T(1.0 - D3Q19::w(0)) * amu : w * amu;
        lvl[i * P.NS + k] = w * (T(1.0 / 3.0) * rho * si);
        lvl[(19 + i) * P.NS + k] = H + w * ph * si;
    }
}

// Fields out: rho, u (Eq. 31), p (Eq. 32) from the level and the phi, mu
// fields of the same time level (any output may be null).
template <class T>
__global__ void k3_fields(const T *__restrict__ lvl, const T *__restrict__ phi,
                          const T *__restrict__ mu, T *rho, T *p, T *ux, T *uy, T *uz,
                          const K3<T> P) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.N) return;
    const Nbr3 n((int)k, P.nx, P.ny, P.nz);
    T f[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = __ldg(lvl + i * P.NS + k);
    const Macro3<T> m = macro3(P, f, phi, mu, n);
    if (rho) rho[k] = m.rho;
    if (p) p[k] = m.p;
    if (ux) ux[k] = m.u[0];
    if (uy) uy[k] = m.u[1];
    if (uz) uz[k] = m.u[2];
}

// Deterministic FP64 partial sums per block (fixed order), then one block
// folds them: out[0] = sum rho, out[1] = sum phi.
template <class T>
__global__ void k3_mass_partial(const T *__restrict__ lvl, double *part, const K3<T> P) {
    __shared__ double sr[256], sp[256];
    double r = 0.0, s = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P.N;
         k += (long long)gridDim.x * blockDim.x) {
        double ph = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) ph += (double)lvl[(19 + i) * P.NS + k];
        s += ph;
        r += (double)P.rhoB + (ph - (double)P.phiB) * (double)P.drho;
    }
    sr[threadIdx.x] = r;
    sp[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sr[threadIdx.x] += sr[threadIdx.x + h];
            sp[threadIdx.x] += sp[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sr[0];
        part[2 * blockIdx.x + 1] = sp[0];
    }
}

// Laplace diagnostic partials: total pressure P = p0 - kappa phi lap phi +
// kappa |grad phi|^2 / 2 + p (Sec. 4.2) summed over r < Rin and r > Rout
// (nearest periodic image), with the counts and the volume of fluid A:
// part[5 b + (0..4)] = sum_in, n_in, sum_out, n_out, volume.
template <class T>
__global__ void k3_laplace_partial(const T *__restrict__ phi, const T *__restrict__ p,
                                   const K3<T> P, double beta, double kappa, double xc, double yc,
                                   double zc, double rin, double rout, double *part) {
    __shared__ double sh[5][256];
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P.N;
         k += (long long)gridDim.x * blockDim.x) {
        const Nbr3 n((int)k, P.nx, P.ny, P.nz);
        const int x = (int)(k % P.nx);
        const int y = (int)((k / P.nx) % P.ny);
        const int z = (int)(k / ((long long)P.nx * P.ny));
        const double ph = (double)phi[k];
        T g[3];
        grad3(phi, n, g);
        const double lp = (double)lap3(phi, n);
        const double pa = (double)P.phiA, pb = (double)P.phiB, pm = 0.5 * (pa + pb);
        const double psi = beta * (ph - pa) * (ph - pa) * (ph - pb) * (ph - pb);
        const double dpsi = 4.0 * beta * (ph - pa) * (ph - pb) * (ph - pm);
        const double gg = (double)g[0] * g[0] + (double)g[1] * g[1] + (double)g[2] * g[2];
        const double Pt = ph * dpsi - psi - kappa * ph * lp + 0.5 * kappa * gg + (double)p[k];
        double dx = fabs(x - xc), dy = fabs(y - yc), dz = fabs(z - zc);
        dx = fmin(dx, P.nx - dx);
        dy = fmin(dy, P.ny - dy);
        dz = fmin(dz, P.nz - dz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < rin) {
            acc[0] += Pt;
            acc[1] += 1.0;
        } else if (r > rout) {
            acc[2] += Pt;
            acc[3] += 1.0;
        }
        acc[4] += (ph - pb) / (pa - pb);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 5; ++j) part[5 * blockIdx.x + j] = sh[j][0];
}

// Folds `nb` partial records of `w` doubles in a fixed order.
__global__ void k3_fold(const double *part, int nb, int w, double *out) {
    if (threadIdx.x < w) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[w * b + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace lbm3
