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
// cells, so 32-bit indices.  Each offset is k plus an x, a y and a z step,
// the steps taking the periodic wrap at the faces.
struct Nbr3 {
    int k;
    int o[19];
    __device__ __forceinline__ Nbr3(int x, int y, int z, int nx, int ny, int nz) { set(x, y, z, nx, ny, nz); }
    __device__ __forceinline__ Nbr3(int kk, int nx, int ny, int nz) {
        const int r = kk / nx;
        set(kk - r * nx, r % ny, r / ny, nx, ny, nz);
    }
    __device__ __forceinline__ void set(int x, int y, int z, int nx, int ny, int nz) {
        const int np = nx * ny;
        k = (z * ny + y) * nx + x;
        const int dx[3] = {x == 0 ? nx - 1 : -1, 0, x == nx - 1 ? 1 - nx : 1};
        const int dy[3] = {y == 0 ? np - nx : -nx, 0, y == ny - 1 ? nx - np : nx};
        const int dz[3] = {z == 0 ? (nz - 1) * np : -np, 0, z == nz - 1 ? (1 - nz) * np : np};
#pragma unroll
        for (int i = 0; i < 19; ++i) o[i] = k + dz[1 + D3Q19::cz(i)] + dy[1 + D3Q19::cy(i)] + dx[1 + D3Q19::cx(i)];
    }
};

// Cell of this thread in the step kernels' launch: x along the block's
// threads, y = blockIdx.y, z = blockIdx.z; false past the x extent.
template <class T>
__device__ __forceinline__ bool cell3(const K3<T> &P, int &x, int &y, int &z) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    return x < P.nx;
}

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
    int x, y, z;
    if (!cell3(P, x, y, z)) return;
    const int k = (z * P.ny + y) * P.nx + x;
    const T *g = lvl + 19 * P.NS + k;
    T s = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) s += __ldg(g + i * P.NS);
    phi[k] = s;
}

template <class T>
__global__ void k3_mu(const T *__restrict__ phi, T *__restrict__ mu, const K3<T> P) {
    int x, y, z;
    if (!cell3(P, x, y, z)) return;
    const Nbr3 n(x, y, z, P.nx, P.ny, P.nz);
    mu[n.k] = mu_of(P, __ldg(phi + n.k), lap3(phi, n));
}

template <class T>
__global__ void k3_p(const T *__restrict__ lvl, const T *__restrict__ phi, const T *__restrict__ mu,
                     T *__restrict__ p, const K3<T> P) {
    int x, y, z;
    if (!cell3(P, x, y, z)) return;
    const Nbr3 n(x, y, z, P.nx, P.ny, P.nz);
    const int k = n.k;
    T f[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = __ldg(lvl + i * P.NS + k);
    p[k] = macro3(P, f, phi, mu, n).p;
}

__device__ __forceinline__ float2 bc3(float a) { return make_float2(a, a); }

// One opposite pair of directions (c, -c) in the two lanes: the
// projections on c (cu = c.u, cF = c.F, cZ = c.F + c.grad(rho)/3,
// cD = c.(grad p - F)) change sign in the second lane; the mu* terms are
// minus the matching u projections.  s = cu (3 + 4.5 cu) - 1.5 u.u (Eq. 26)
// and the f, g collisions of Eqs. 22-29 with Gamma = 1 + s.
__device__ __forceinline__ void collide_pair3(float2 cu, float2 cF, float2 cZ, float2 cD, float w,
                                              float2 mu15, float2 muF, float2 muZ, float2 muD,
                                              float2 Kf, float2 Bf, float2 pf, float2 omf, float2 Ag,
                                              float2 phg, float2 Q, float2 omg, float2 f, float2 g,
                                              float2 &fo, float2 &go) {
    const float2 sg = make_float2(1.0f, -1.0f);
    const float2 si = __ffma2_rn(cu, __ffma2_rn(cu, bc3(4.5f), make_float2(3.0f, -3.0f)), mu15);
    const float2 eF = __ffma2_rn(cF, sg, muF);
    const float2 eZ = __ffma2_rn(cZ, sg, muZ);
    const float2 eD = __ffma2_rn(cD, sg, muD);
    const float2 w2 = bc3(w);
    float2 a = __ffma2_rn(Bf, si, Kf);
    a = __ffma2_rn(pf, __ffma2_rn(si, eZ, eF), a);
    fo = __ffma2_rn(omf, f, __fmul2_rn(w2, a));
    float2 b = __ffma2_rn(phg, si, Ag);
    b = __ffma2_rn(Q, __ffma2_rn(si, eD, eD), b);
    go = __ffma2_rn(omg, g, __fmul2_rn(w2, b));
}

// Pass 4: collision (Eqs. 22-29, Gamma_i = 1 + s_i) and push.  FP32 is
// held to 128 registers (16 warps per SM; left free it took 144 and ran
// 20% slower).
template <class T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k3_collide(const T *__restrict__ src, T *__restrict__ dst, const T *__restrict__ phi,
                           const T *__restrict__ mu, const T *__restrict__ pf_, const K3<T> P) {
    int x, y, z;
    if (!cell3(P, x, y, z)) return;
    const Nbr3 n(x, y, z, P.nx, P.ny, P.nz);
    const int k = n.k;
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
    if constexpr (sizeof(T) == 4) {
        // FP32: rest direction, then the 9 opposite pairs (2j-1, 2j) in
        // packed f32x2 arithmetic (collide_pair3)
        const float uZ = uF + (1.0f / 3.0f) * uR;
        {
            const float si = -uu15, eF = -uF, eZ = -uZ, eD = -uD, w = float(D3Q19::w(0));
            const float fv = omf * f[0] + w * (Kf + Bf * si + P.pf * (eF + si * eZ));
            const float Hg = (phg - float(1.0 - D3Q19::w(0)) * Ag) * float(1.0 / D3Q19::w(0));
            const float gv = omg * g[0] + w * (Hg + phg * si + Q * (eD + si * eD));
            dst[k] = fv;
            dst[19 * P.NS + k] = gv;
        }
        const float2 mu15 = bc3(-uu15), muF = bc3(-uF), muZ = bc3(-uZ), muD = bc3(-uD);
        const float2 Kf2 = bc3(Kf), Bf2 = bc3(Bf), pf2 = bc3(P.pf), omf2 = bc3(omf);
        const float2 Ag2 = bc3(Ag), phg2 = bc3(phg), Q2 = bc3(Q), omg2 = bc3(omg);
#pragma unroll
        for (int i = 1; i < 19; i += 2) {
            const float cx = float(D3Q19::cx(i)), cy = float(D3Q19::cy(i)), cz = float(D3Q19::cz(i));
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cF = cx * m.F[0] + cy * m.F[1] + cz * m.F[2];
            const float cZ = cF + (1.0f / 3.0f) * (cx * gr[0] + cy * gr[1] + cz * gr[2]);
            const float cD = cx * D[0] + cy * D[1] + cz * D[2];
            float2 fo, go;
            collide_pair3(bc3(cu), bc3(cF), bc3(cZ), bc3(cD), float(D3Q19::w(i)), mu15, muF, muZ, muD, Kf2,
                          Bf2, pf2, omf2, Ag2, phg2, Q2, omg2, make_float2(f[i], f[i + 1]),
                          make_float2(g[i], g[i + 1]), fo, go);
            dst[i * P.NS + n.o[i]] = fo.x;
            dst[(i + 1) * P.NS + n.o[i + 1]] = fo.y;
            dst[(19 + i) * P.NS + n.o[i]] = go.x;
            dst[(20 + i) * P.NS + n.o[i + 1]] = go.y;
        }
    } else {
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
__global__ void __launch_bounds__(256) k3_mass_partial(const T *__restrict__ lvl, double *part, const K3<T> P) {
    __shared__ double sr[8], sp[8];
    double r = 0.0, s = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P.N;
         k += (long long)gridDim.x * blockDim.x) {
        double ph = 0.0;
#pragma unroll
        for (int i = 0; i < 19; ++i) ph += (double)lvl[(19 + i) * P.NS + k];
        s += ph;
        r += (double)P.rhoB + (ph - (double)P.phiB) * (double)P.drho;
    }
    // warp shuffles, then the 8 warp sums in order: a fixed summation order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r += __shfl_down_sync(0xffffffffu, r, o);
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sr[wid] = r;
        sp[wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 8; ++i) {
            a += sr[i];
            b += sp[i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// Laplace diagnostic partials: total pressure P = p0 - kappa phi lap phi +
// kappa |grad phi|^2 / 2 + p (Sec. 4.2) summed over r < Rin and r > Rout
// (nearest periodic image), with the counts and the volume of fluid A:
// part[5 b + (0..4)] = sum_in, n_in, sum_out, n_out, volume.
template <class T>
__global__ void __launch_bounds__(256) k3_laplace_partial(const T *__restrict__ phi, const T *__restrict__ p,
                                   const K3<T> P, double beta, double kappa, double xc, double yc,
                                   double zc, double rin, double rout, double *part) {
    __shared__ double sh[5][8];
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
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 5; ++j) sh[j][wid] = acc[j];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            double a = 0.0;
            for (int i = 0; i < 8; ++i) a += sh[j][i];
            part[5 * blockIdx.x + j] = a;
        }
}

// Folds `nb` partial records of `w` (<= 8) doubles in a fixed order, one
// block of 256 threads: thread t sums records t, t + 256, ... in ascending
// order, each warp folds its sums by shuffles, thread j adds the 8 warp
// sums of total j in warp order.
__global__ void __launch_bounds__(256) k3_fold(const double *part, int nb, int w, double *out) {
    __shared__ double ws[8][8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int j = 0; j < w; ++j) {
        double a = 0.0;
        for (int b = t; b < nb; b += 256) a += part[w * b + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) ws[wid][j] = a;
    }
    __syncthreads();
    if (t < w) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += ws[k][t];
        out[t] = s;
    }
}

}  // namespace lbm3
