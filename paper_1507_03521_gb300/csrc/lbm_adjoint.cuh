// lbm_adjoint.cuh — hand-written discrete adjoint (vector-Jacobian product)
// of one time step, of the equilibrium initial state and of the loss
// L = sum (phi_T - phi_target)^2, for FP64 / FP32 populations in the plain
// layout.
//
// With s_t the populations at step t and lambda_t = dL/ds_t:
//   lambda_t = (d s_{t+1} / d s_t)^T lambda_{t+1},
//   dL/dM, dL/dsigma += (d s_{t+1} / d(M, sigma))^T lambda_{t+1}.
// The forward step (Sec. 3) is a chain of local maps and stencils:
//   phi = sum g, rho(phi)            (Eqs. 30, 11)
//   mu = psi'(phi) - kappa lap phi   (Eq. 5)
//   grad phi, grad mu, lap mu; F; u; p (Eqs. 31-32)
//   grad p; collision (Eqs. 22-29); streaming / bounce-back.
// The adjoint runs the chain backwards.  Local maps are differentiated by
// hand; every stencil is applied transposed as a gather (each cell collects
// from the cells whose stencils read it, with the ghost-row rules of the
// forward step: mirror for phi and mu, linear extrapolation for p), so the
// result is deterministic.  Kernels, in order, for one reverse step:
//   k_step<MODE_ADJC>     the forward fields of step t, recomputed on tiles
//                         with halos as the forward tile step does
//                         (lbm_kernels.cuh), then streaming and collision
//                         transposed per cell (AdjCell, adj_collide_cell),
//   k_adj_p               grad p transposed, then u, p, F backwards,
//   k_adj_muphi           grad mu and lap mu transposed, then grad phi and
//                         lap phi transposed and phi = sum g, per tile; the
//                         step's (M, sigma) sums, folded by its last CTA,
//   k_adj_theta           per-cell (M, sigma) terms reduced in FP64 (the
//                         initial state's; a step's come from k_adj_muphi).
// M enters through alpha = M / (cs2 (tau_g - 1/2)) and gamma lambda with
// lambda = M (Eq. 33); sigma through kappa and beta, both proportional to
// sigma (Eqs. 3-4 solved), so mu = sigma mu1.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class T>
struct AdjP {
    KP<T> k;
    T alpha1;  // alpha per unit M
    T gamma;   // gamma (Eq. 17)
    T kappa1, beta1;  // kappa, beta per unit sigma
};

// Work arrays of the adjoint, each N (padded NS) elements of T.
enum AdjArr {
    A_PHI, A_RHO, A_MU, A_MU1, A_GPHX, A_GPHY, A_GMUX, A_GMUY, A_LMU, A_FX, A_FY, A_UX, A_UY,
    A_P, A_GPX, A_GPY,
    B_P, B_RHO, B_PHI, B_MU, B_UX, B_UY, B_FX, B_FY, B_GRX, B_GRY, B_LMU, B_GPX, B_GPY,
    B_GPHX, B_GPHY, B_GMUX, B_GMUY, B_ALPHA, B_GL, B_SIGMA,
    A_COUNT
};


template <class T>
struct AdjW {
    T *a;          // A_COUNT arrays of NS elements
    long long NS;
    __device__ __forceinline__ T *operator[](int k) const { return a + (long long)k * NS; }
};

// ------------------------------------------------------------- helpers

template <class T>
struct Nb {
    int nx, ny, wall;
    // periodic x
    __device__ __forceinline__ int wx(int x) const { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
    // row of a stencil read at row y: periodic wrap or mirror
    __device__ __forceinline__ int my(int y) const {
        if (!wall) return y < 0 ? y + ny : (y >= ny ? y - ny : y);
        return y < 0 ? -y - 1 : (y >= ny ? 2 * ny - 1 - y : y);
    }
};

// Forward isotropic gradient / Laplacian at (x, y) of a global array with
// mirror ghosts (extrap = false) or linear-extrapolation ghosts (p).
template <class T>
__device__ __forceinline__ T nbval(const T *v, const Nb<T> &B, int x, int y, bool extrap) {
    const int xx = B.wx(x);
    if (!B.wall || (y >= 0 && y < B.ny)) return v[(long long)B.my(y) * B.nx + xx];
    if (!extrap) return v[(long long)B.my(y) * B.nx + xx];
    if (y < 0) return T(2) * v[xx] - v[(long long)B.nx + xx];
    return T(2) * v[(long long)(B.ny - 1) * B.nx + xx] - v[(long long)(B.ny - 2) * B.nx + xx];
}

template <class T>
__device__ __forceinline__ void grad_g(const T *v, const Nb<T> &B, int x, int y, bool extrap, T &gx,
                                       T &gy) {
    T sx = T(0), sy = T(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const T n = nbval(v, B, x + D2Q9::cx(i), y + D2Q9::cy(i), extrap);
        sx += T(3.0 * D2Q9::w(i) * D2Q9::cx(i)) * n;
        sy += T(3.0 * D2Q9::w(i) * D2Q9::cy(i)) * n;
    }
    gx = sx;
    gy = sy;
}

template <class T>
__device__ __forceinline__ T lap_g(const T *v, const Nb<T> &B, int x, int y) {
    const T c = v[(long long)y * B.nx + x];
    T acc = T(0);
#pragma unroll
    for (int i = 1; i < 9; ++i)
        acc += T(6.0 * D2Q9::w(i)) * (nbval(v, B, x + D2Q9::cx(i), y + D2Q9::cy(i), false) - c);
    return acc;
}

// Transposed stencil as a gather at target (x, y): the sum over every
// (centre c, direction i) whose forward read of direction i lands on the
// target, of coef * term(c, i); coef follows the ghost rule (1 for a direct
// or mirrored read; 2 and -1 for the two rows an extrapolated ghost uses).
template <class T, class F>
__device__ __forceinline__ T tgather(const Nb<T> &B, int x, int y, bool extrap, F &&term) {
    T acc = T(0);
    const int nx = B.nx, ny = B.ny;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
        const int sx = B.wx(x - cx);
        int sy = y - cy;
        if (!B.wall) {
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            acc += term((long long)sy * nx + sx, i, T(1));
            continue;
        }
        if (sy >= 0 && sy < ny) acc += term((long long)sy * nx + sx, i, T(1));
        // ghost reads: centre on the edge row, direction pointing out of it
        if (cy == -1) {
            if (!extrap) {
                if (y == 0) acc += term((long long)sx, i, T(1));
            } else {
                if (y == 0) acc += term((long long)sx, i, T(2));
                if (y == 1) acc += term((long long)sx, i, T(-1));
            }
        } else if (cy == 1) {
            const long long top = (long long)(ny - 1) * nx + sx;
            if (!extrap) {
                if (y == ny - 1) acc += term(top, i, T(1));
            } else {
                if (y == ny - 1) acc += term(top, i, T(2));
                if (y == ny - 2) acc += term(top, i, T(-1));
            }
        }
    }
    return acc;
}

// x mod n in [0, n), for any x
__device__ __forceinline__ int adj_wrap(int x, int n) {
    x %= n;
    return x < 0 ? x + n : x;
}

#define ADJ_LOOP(k, N)                                                            \
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (N); \
         k += (long long)gridDim.x * blockDim.x)

// Row of cell k (row length nx): a 32-bit division whenever k fits in an
// int (every grid below 2^31 cells), the 64-bit one otherwise.
__device__ __forceinline__ int row_of(long long k, int nx) {
    return k <= 0x7fffffffLL ? (int)k / nx : (int)(k / nx);
}

// -------------------------------------- forward fields of the initial state

// phi given directly (initial state): copy into A_PHI.
template <class T>
__global__ void k_adj_phi0(const T *__restrict__ phi0, const AdjP<T> P, AdjW<T> W) {
    const long long N = (long long)P.k.nx * P.k.ny;
    ADJ_LOOP(k, N) W[A_PHI][k] = phi0[k];
}

// mu, mu per unit sigma, grad phi.
template <class T>
__global__ void k_adj_f1(const AdjP<T> P, AdjW<T> W) {
    const Nb<T> B{P.k.nx, P.k.ny, P.k.wall};
    const long long N = (long long)P.k.nx * P.k.ny;
    ADJ_LOOP(k, N) {
        const int y = row_of(k, B.nx), x = (int)(k - (long long)y * B.nx);
        const T ph = W[A_PHI][k];
        const T lap = lap_g(W[A_PHI], B, x, y);
        const T q = (ph - P.k.phiA) * (ph - P.k.phiB) * (ph - P.k.phibar);
        W[A_MU][k] = P.k.beta4 * q - P.k.kappa * lap;
        W[A_MU1][k] = T(4) * P.beta1 * q - P.kappa1 * lap;
        T gx, gy;
        grad_g(W[A_PHI], B, x, y, false, gx, gy);
        W[A_GPHX][k] = gx;
        W[A_GPHY][k] = gy;
    }
}

// ------------------------------------------------------------ reverse

// Streaming and collision transposed at cell k = (x, y), about the forward
// fields of the step: lambda_t's direct (1 - 1/tau) terms from lam_next
// (lambda_{t+1}; k_adj_p and k_adj_muphi add the terms through p, j and
// phi) and the adjoints of the fields the collision reads (B_* arrays).
template <class T>
__device__ __forceinline__ void adj_collide_cell(const KP<T> &K, int x, int y, long long k, T phi, T rho,
                                                 T mu, T p, T ux, T uy, T Fx, T Fy, T gphx, T gphy,
                                                 T lm, T gpx, T gpy, const T *__restrict__ lam_next,
                                                 T *__restrict__ lam, const AdjW<T> &W) {
    const Nb<T> B{K.nx, K.ny, K.wall};
    const long long NS = K.NS;
    const T grx = K.drho * gphx, gry = K.drho * gphy;
    const T uu = ux * ux + uy * uy;
    const T q = -T(3) * phi / rho;
    // per-cell quotients, hoisted out of the direction loop (divisions
    // are many instructions each; by 3 they become a multiply by 1/3)
    const T c13 = T(1.0 / 3.0);
    const T rho3 = rho * c13, grx3 = grx * c13, gry3 = gry * c13;
    const T m3r = -T(3) / rho, p3r2 = T(3) * phi / (rho * rho);
    const T Dx = gpx - Fx, Dy = gpy - Fy;
    T bp = 0, brho = 0, bphi = 0, bmu = 0, bux = 0, buy = 0, bFx = 0, bFy = 0, bgrx = 0,
      bgry = 0, blm = 0, bgpx = 0, bgpy = 0, balpha = 0, bgl = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
        const T w = T(D2Q9::w(i));
        // lambda of the post-collision population: where streaming put it
        const int yd = y + cy;
        T lf, lg;
        if (B.wall && (yd < 0 || yd >= B.ny)) {
            const int o = D2Q9::opp(i);
            lf = lam_next[o * NS + k];
            lg = lam_next[(9 + o) * NS + k];
            const T cuw = T(cx) * (yd < 0 ? K.uwb : K.uwt);
            brho += -T(2) * w * cuw * lf;   // f_opp = f*_i - 2 w rho c.u_w
            bphi += -T(6) * w * cuw * lg;   // g_opp = g*_i - 2 w phi c.u_w / cs2
        } else {
            const int xx = B.wx(x + cx);
            const int yy = yd < 0 ? yd + B.ny : (yd >= B.ny ? yd - B.ny : yd);
            const long long kd = (long long)yy * B.nx + xx;
            lf = lam_next[i * NS + kd];
            lg = lam_next[(9 + i) * NS + kd];
        }
        lam[i * NS + k] = (T(1) - K.itf) * lf;
        lam[(9 + i) * NS + k] = (T(1) - K.itg) * lg;
        const T beq = K.itf * lf, bF = K.pf * lf;    // d/d f^eq_i, d/d F_i
        const T bgeq = K.itg * lg, bG = K.pg * lg;   // d/d g^eq_i, d/d G_i
        const T cu = T(cx) * ux + T(cy) * uy;
        const T s = T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
        const T ex = T(cx) - ux, ey = T(cy) - uy;
        T bs = 0;
        // f^eq_i = w (p + rho s / 3)   (Eq. 24)
        bp += w * beq;
        brho += w * s * c13 * beq;
        bs += w * rho3 * beq;
        // g^eq_i = H_i + w phi s   (Eqs. 25, 27)
        if (i == 0) {
            bphi += bgeq;
            bmu += -T(1.0 - D2Q9::w(0)) * K.alpha * bgeq;
            balpha += -T(1.0 - D2Q9::w(0)) * mu * bgeq;
        } else {
            bmu += w * K.alpha * bgeq;
            balpha += w * mu * bgeq;
        }
        bphi += w * s * bgeq;
        bs += w * phi * bgeq;
        // F_i = (c - u).[w (1 + s) F + w s grad rho / 3] - w rho gamma lambda lap mu / 3
        const T eF = ex * Fx + ey * Fy, eR = ex * grx + ey * gry;
        const T Ax = w * (T(1) + s) * Fx + w * s * grx3;
        const T Ay = w * (T(1) + s) * Fy + w * s * gry3;
        bFx += w * (T(1) + s) * ex * bF;
        bFy += w * (T(1) + s) * ey * bF;
        bgrx += w * s * c13 * ex * bF;
        bgry += w * s * c13 * ey * bF;
        bs += w * (eF + eR * c13) * bF;
        bux += -Ax * bF;
        buy += -Ay * bF;
        brho += -w / T(3) * K.gl * lm * bF;
        blm += -w / T(3) * rho * K.gl * bF;
        bgl += -w / T(3) * rho * lm * bF;
        // G_i = q w (1 + s) (c - u).(grad p - F), q = -phi / (cs2 rho)
        const T E = ex * Dx + ey * Dy;
        const T wg = w * (T(1) + s);
        bphi += m3r * wg * E * bG;
        brho += p3r2 * wg * E * bG;
        bs += q * w * E * bG;
        bux += -q * wg * Dx * bG;
        buy += -q * wg * Dy * bG;
        bgpx += q * wg * ex * bG;
        bgpy += q * wg * ey * bG;
        bFx += -q * wg * ex * bG;
        bFy += -q * wg * ey * bG;
        // s_i = 3 c.u + 4.5 (c.u)^2 - 1.5 |u|^2   (Eq. 26)
        bux += bs * (T(3) * T(cx) + T(9) * cu * T(cx) - T(3) * ux);
        buy += bs * (T(3) * T(cy) + T(9) * cu * T(cy) - T(3) * uy);
    }
    W[B_P][k] = bp;
    W[B_RHO][k] = brho;
    W[B_PHI][k] = bphi;
    W[B_MU][k] = bmu;
    W[B_UX][k] = bux;
    W[B_UY][k] = buy;
    W[B_FX][k] = bFx;
    W[B_FY][k] = bFy;
    W[B_GRX][k] = bgrx;
    W[B_GRY][k] = bgry;
    W[B_LMU][k] = blm;
    W[B_GPX][k] = bgpx;
    W[B_GPY][k] = bgpy;
    W[B_ALPHA][k] = balpha;
    W[B_GL][k] = bgl;
}

// MODE_ADJC of the tile kernel (k_step): per owned cell, the forward fields
// the later reverse kernels read (k_adj_p: phi, rho, lap mu, u, grad phi,
// grad mu; k_adj_muphi: phi, mu per unit sigma), then the collision
// adjoint about all of them, in the same thread.
template <class T>
struct AdjCell {
    static __device__ __forceinline__ void run(const KP<T> &K, const FieldOut<T> &out, int x, int y,
                                               long long k, const Macro<T> &m, T mu1, T p, T gpx,
                                               T gpy) {
        const AdjW<T> W{out.adj, out.adj_ns};
        W[A_PHI][k] = m.phi;
        W[A_RHO][k] = m.rho;
        W[A_MU1][k] = mu1;
        W[A_GPHX][k] = m.gphx;
        W[A_GPHY][k] = m.gphy;
        W[A_GMUX][k] = m.gmux;
        W[A_GMUY][k] = m.gmuy;
        W[A_LMU][k] = m.lmu;
        W[A_UX][k] = m.ux;
        W[A_UY][k] = m.uy;
        adj_collide_cell(K, x, y, k, m.phi, m.rho, m.mu, p, m.ux, m.uy, m.Fx, m.Fy, m.gphx, m.gphy,
                         m.lmu, gpx, gpy, out.lam_next, out.lam, W);
    }
};

// grad p transposed (extrapolated ghosts) gives the full adjoint of p; then
// p, u, F backwards (Eqs. 31-32) and the f terms through sum f and j.
// FP32: 3 CTAs per SM (80 registers).  With every load of a cell before
// its first store, 4 CTAs per SM (64 registers) spill 128 bytes and the
// whole backward pass at 512^2 measured 2.4% slower.
template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_adj_p(T *__restrict__ lam, const AdjP<T> P, AdjW<T> W) {
    const Nb<T> B{P.k.nx, P.k.ny, P.k.wall};
    const long long N = (long long)P.k.nx * P.k.ny, NS = P.k.NS;
    const KP<T> &K = P.k;
    const T *gbx = W[B_GPX], *gby = W[B_GPY];
    ADJ_LOOP(k, N) {
        const int y = row_of(k, B.nx), x = (int)(k - (long long)y * B.nx);
        // Every load of the cell comes before its first store: the work
        // arrays and lambda are views of allocations the compiler cannot
        // tell apart, so a load placed after a store would wait for it,
        // one L2 round trip after another.
        const T bp = W[B_P][k] + tgather(B, x, y, true, [&](long long c, int i, T coef) {
                         return coef * T(3.0 * D2Q9::w(i)) *
                                (T(D2Q9::cx(i)) * gbx[c] + T(D2Q9::cy(i)) * gby[c]);
                     });
        const T rho = W[A_RHO][k], phi = W[A_PHI][k], lm = W[A_LMU][k];
        const T ux = W[A_UX][k], uy = W[A_UY][k];
        const T gphx = W[A_GPHX][k], gphy = W[A_GPHY][k];
        const T gmux = W[A_GMUX][k], gmuy = W[A_GMUY][k];
        const T bux0 = W[B_UX][k], buy0 = W[B_UY][k], bgrx = W[B_GRX][k], bgry = W[B_GRY][k];
        const T blm0 = W[B_LMU][k], brho0 = W[B_RHO][k], bgl0 = W[B_GL][k];
        const T bFx0 = W[B_FX][k], bFy0 = W[B_FY][k], bphi0 = W[B_PHI][k];
        T l[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) l[i] = lam[i * NS + k];
        // p = sum f + (drho u.grad phi - gamma lambda rho lap mu) / 6
        const T bux = bux0 + K.drho / T(6) * gphx * bp;
        const T buy = buy0 + K.drho / T(6) * gphy * bp;
        const T bgphx = K.drho / T(6) * ux * bp + K.drho * bgrx;
        const T bgphy = K.drho / T(6) * uy * bp + K.drho * bgry;
        const T blm = blm0 - K.gl / T(6) * rho * bp;
        T brho = brho0 - K.gl / T(6) * lm * bp;
        const T bgl = bgl0 + -rho * lm / T(6) * bp;
        // u = (j + F/6) 3 / rho
        const T jx = T(3) / rho * bux, jy = T(3) / rho * buy;
        const T bFx = bFx0 + bux / (T(2) * rho);
        const T bFy = bFy0 + buy / (T(2) * rho);
        brho += -(ux * bux + uy * buy) / rho;
        // F = -phi grad mu + (0, -(rho - rho_ref) g)
        brho += -K.grav * bFy;
        W[B_GL][k] = bgl;
        W[B_PHI][k] = bphi0 + -(gmux * bFx + gmuy * bFy);
        W[B_GMUX][k] = -phi * bFx;
        W[B_GMUY][k] = -phi * bFy;
        W[B_GPHX][k] = bgphx;
        W[B_GPHY][k] = bgphy;
        W[B_LMU][k] = blm;
        W[B_RHO][k] = brho;
        // sum f and j feed every f_i
#pragma unroll
        for (int i = 0; i < 9; ++i)
            lam[i * NS + k] = l[i] + (bp + T(D2Q9::cx(i)) * jx + T(D2Q9::cy(i)) * jy);
    }
}

// Block partial sums of the (M, sigma) terms, in a fixed order: each
// thread's grid-stride sums, warp shuffles, then the 8 warp sums in order
// (one block of 256 threads).
__device__ __forceinline__ void adj_theta_partials(double dM, double dS, double *__restrict__ part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dM += __shfl_down_sync(0xffffffffu, dM, o);
        dS += __shfl_down_sync(0xffffffffu, dS, o);
    }
    __shared__ double wm[8], ws[8];
    if ((threadIdx.x & 31) == 0) {
        wm[threadIdx.x >> 5] = dM;
        ws[threadIdx.x >> 5] = dS;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 8; ++i) {
            a += wm[i];
            b += ws[i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// The mu and phi adjoints of a reverse step, and the fold of its (M, sigma)
// partial sums, in one launch.  A CTA of 256 threads takes
// 64 x 8 tiles in turn: it computes mu_bar on the tile and a ring of one
// cell into shared memory (the ring cells are recomputed by each
// neighbouring tile and only read here), then the phi adjoint of the tile
// from it.  Its inputs are final before the launch; its global writes are
// the tile cells' lambda_t g slots and the CTA's (M, sigma) partial sums.
// The last CTA to finish (a ticket counter; the counter is left at zero)
// folds the partial sums into the running totals, in the same fixed order
// as k_adj_accumulate.  64-column tiles, two cells per thread: a 512^2
// grid has 512 tiles, all resident at once (with 32-column tiles its 1024
// tiles took two rounds of the 608 CTAs the partial sums allow).  FP32:
// held to 4 CTAs per SM (64 registers, no spill) so that those 512 tiles
// stay resident at once.
constexpr int kMpTX = 64, kMpTY = 8;

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_adj_muphi(T *__restrict__ lam, const AdjP<T> P, AdjW<T> W,
                                                   double *__restrict__ part, double *__restrict__ acc,
                                                   unsigned *__restrict__ ticket) {
    constexpr int HX = kMpTX + 2, HY = kMpTY + 2;
    // mu_bar and the grad phi adjoint on the tile and its ring
    __shared__ T smu[HY][HX], sgx[HY][HX], sgy[HY][HX];
    __shared__ bool last;
    const Nb<T> B{P.k.nx, P.k.ny, P.k.wall};
    const KP<T> &K = P.k;
    const long long NS = K.NS;
    const int nx = B.nx, ny = B.ny;
    const int tid = threadIdx.x;  // 1-D block of 256
    const int tilesx = (nx + kMpTX - 1) / kMpTX, tilesy = (ny + kMpTY - 1) / kMpTY;
    const long long ntiles = (long long)tilesx * tilesy;
    const T *gmx = W[B_GMUX], *gmy = W[B_GMUY], *bl = W[B_LMU];
    const T *gpx = W[B_GPHX], *gpy = W[B_GPHY];
    const double a1 = (double)P.alpha1, gm = (double)P.gamma;
    double dM = 0.0, dS = 0.0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx0 = (int)(tile % tilesx) * kMpTX, ty0 = (int)(tile / tilesx) * kMpTY;
        // mu_bar on the tile and its ring: grad mu and lap mu transposed
        for (int j = tid; j < HX * HY; j += 256) {
            const int hx = j % HX, hy = j / HX;
            const int xv = tx0 - 1 + hx, yv = ty0 - 1 + hy;
            if (B.wall && (yv < 0 || yv >= ny)) continue;
            const int x = adj_wrap(xv, nx), y = B.wall ? yv : adj_wrap(yv, ny);
            const long long k = (long long)y * nx + x;
            const T t = tgather(B, x, y, false, [&](long long c, int i, T coef) {
                return coef * (T(3.0 * D2Q9::w(i)) * (T(D2Q9::cx(i)) * gmx[c] + T(D2Q9::cy(i)) * gmy[c]) +
                               T(6.0 * D2Q9::w(i)) * bl[c]);
            });
            const T bmu = W[B_MU][k] + t - T(10.0 / 3.0) * bl[k];
            smu[hy][hx] = bmu;
            sgx[hy][hx] = gpx[k];
            sgy[hy][hx] = gpy[k];
            if (hx >= 1 && hx <= kMpTX && hy >= 1 && hy <= kMpTY && xv < nx && yv < ny) {
                dM += a1 * (double)W[B_ALPHA][k] + gm * (double)W[B_GL][k];
                dS += (double)(bmu * W[A_MU1][k]);
            }
        }
        __syncthreads();
        // phi adjoint of the tile: grad phi and lap phi transposed, phi = sum g
        for (int j = tid; j < kMpTX * kMpTY; j += 256) {
            const int lx = j % kMpTX, ly = j / kMpTX;
            const int x = tx0 + lx, y = ty0 + ly;
            if (x >= nx || y >= ny) continue;
            const long long k = (long long)y * nx + x;
            const int sx0 = lx + 1, sy0 = ly + 1;
            const T ph = W[A_PHI][k];
            const T a = ph - K.phiA, b = ph - K.phiB, m = ph - K.phibar;
            const T psi2 = K.beta4 * (a * b + a * m + b * m);
            // tgather's terms in its order; mu_bar and the grad phi adjoint
            // of a source centre from shared memory (the centre's tile
            // position, which the first phase filled from cell c)
            auto term = [&](long long c, int hx, int hy, int i, T coef) {
                (void)c;
                return coef * (T(3.0 * D2Q9::w(i)) * (T(D2Q9::cx(i)) * sgx[hy][hx] + T(D2Q9::cy(i)) * sgy[hy][hx]) -
                               K.kappa * T(6.0 * D2Q9::w(i)) * smu[hy][hx]);
            };
            T t = T(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
                const int sx = B.wx(x - cx), hx = sx0 - cx;
                int sy = y - cy;
                if (!B.wall) {
                    sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                    t += term((long long)sy * nx + sx, hx, sy0 - cy, i, T(1));
                    continue;
                }
                if (sy >= 0 && sy < ny) t += term((long long)sy * nx + sx, hx, sy0 - cy, i, T(1));
                if (cy == -1 && y == 0) t += term((long long)sx, hx, sy0, i, T(1));
                if (cy == 1 && y == ny - 1) t += term((long long)(ny - 1) * nx + sx, hx, sy0, i, T(1));
            }
            const T bm = smu[sy0][sx0];
            const T bphi = W[B_PHI][k] + K.drho * W[B_RHO][k] + psi2 * bm + t + K.kappa * T(10.0 / 3.0) * bm;
            // the nine loads before the nine stores (see k_adj_p)
            T l[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) l[i] = lam[(9 + i) * NS + k];
#pragma unroll
            for (int i = 0; i < 9; ++i) lam[(9 + i) * NS + k] = l[i] + bphi;
        }
        __syncthreads();
    }
    adj_theta_partials(dM, dS, part);
    // the last CTA folds every CTA's partial sums
    __threadfence();
    if (tid == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        fold_partials<true>(part, gridDim.x, 2, acc);
        if (tid == 0) *ticket = 0u;
    }
}

// Adjoint of the equilibrium initial state (u = 0: f = 0, g_0 = phi -
// (1 - w_0) alpha mu, g_i = w_i alpha mu): mu_bar, alpha_bar and sigma_bar
// per cell, from lambda_0 (g slots).
template <class T>
__global__ void k_adj_init_a(const T *__restrict__ lam0, const AdjP<T> P, AdjW<T> W) {
    const long long N = (long long)P.k.nx * P.k.ny, NS = P.k.NS;
    ADJ_LOOP(k, N) {
        T br = -T(1.0 - D2Q9::w(0)) * lam0[9 * NS + k];
#pragma unroll
        for (int i = 1; i < 9; ++i) br += T(D2Q9::w(i)) * lam0[(9 + i) * NS + k];
        const T bmu = P.k.alpha * br;
        W[B_MU][k] = bmu;
        W[B_ALPHA][k] = W[A_MU][k] * br;
        W[B_GL][k] = T(0);
        W[B_SIGMA][k] = bmu * W[A_MU1][k];
    }
}

// phi0_bar = lambda_0 g_0 + psi'' mu_bar - kappa lap^T mu_bar.
template <class T>
__global__ void k_adj_init_b(const T *__restrict__ lam0, T *__restrict__ phi0_bar, const AdjP<T> P,
                             AdjW<T> W) {
    const Nb<T> B{P.k.nx, P.k.ny, P.k.wall};
    const long long N = (long long)P.k.nx * P.k.ny, NS = P.k.NS;
    const KP<T> &K = P.k;
    const T *bm = W[B_MU];
    ADJ_LOOP(k, N) {
        const int y = row_of(k, B.nx), x = (int)(k - (long long)y * B.nx);
        const T ph = W[A_PHI][k];
        const T a = ph - K.phiA, b = ph - K.phiB, m = ph - K.phibar;
        const T psi2 = K.beta4 * (a * b + a * m + b * m);
        const T t = tgather(B, x, y, false, [&](long long c, int i, T coef) {
            return coef * (-K.kappa * T(6.0 * D2Q9::w(i)) * bm[c]);
        });
        phi0_bar[k] = lam0[9 * NS + k] + psi2 * bm[k] + t + K.kappa * T(10.0 / 3.0) * bm[k];
    }
}

// Loss seed: lambda_T = dL/ds_T with L = sum (phi_T - target)^2; per-block
// FP64 partial sums of the loss.
template <class T>
__global__ void __launch_bounds__(256)
k_adj_seed(const T *__restrict__ lvl, const T *__restrict__ target, T *__restrict__ lam,
           const AdjP<T> P, double *__restrict__ part) {
    const long long N = (long long)P.k.nx * P.k.ny, NS = P.k.NS;
    double acc = 0.0;
    ADJ_LOOP(k, N) {
        T phi = T(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) phi += lvl[(9 + i) * NS + k];
        const T d = phi - target[k];
        acc += (double)d * (double)d;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lam[i * NS + k] = T(0);
            lam[(9 + i) * NS + k] = T(2) * d;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double wsum[8];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < 8; ++i) a += wsum[i];
        part[blockIdx.x] = a;
    }
}

// Per-block FP64 partial sums of the (M, sigma) terms of one reverse step:
// dM = sum alpha1 alpha_bar + gamma (gamma lambda)_bar, dsigma = sum sigma_bar.
template <class T>
__global__ void __launch_bounds__(256)
k_adj_theta(const AdjP<T> P, AdjW<T> W, double *__restrict__ part) {
    const long long N = (long long)P.k.nx * P.k.ny;
    double dM = 0.0, dS = 0.0;
    const double a1 = (double)P.alpha1, gm = (double)P.gamma;
    ADJ_LOOP(k, N) {
        dM += a1 * (double)W[B_ALPHA][k] + gm * (double)W[B_GL][k];
        dS += (double)W[B_SIGMA][k];
    }
    adj_theta_partials(dM, dS, part);
}

// Adds the per-block partials (fold_partials order) to the running totals.
static __global__ void __launch_bounds__(256) k_adj_accumulate(const double *__restrict__ part, int nblocks,
                                                               int width, double *__restrict__ acc) {
    fold_partials<true>(part, nblocks, width, acc);
}

}  // namespace lbm
