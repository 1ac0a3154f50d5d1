// lbm_strip.cuh — the streaming form of the time step, for grids whose nx
// is a multiple of 8.
//
// Same arithmetic as k_step (lbm_kernels.cuh), reorganised so that the
// radius-3 coupling of the step (grad p <- p <- lap mu <- lap phi) costs
// an x-halo only:
//   * A CTA of SW threads owns a column strip x0 .. x0+SW-1 and a segment
//     of rows ys .. ye-1, and marches up through y.  Iteration y
//       1. phi       at row y+3 from the g populations of that row,
//       2. sum f, j  at row y+1 from the f populations of that row,
//       3. mu        at row y+2 (Eq. 5),
//       4. u, p, F, lap mu, grad phi at row y+1 (Eqs. 31-32),
//       5. collides row y (Eqs. 22-29) and pushes it to the other level.
//     Rows of phi, mu, p and u live in small shared-memory rings.
//   * Population rows are copied global -> shared with cp.async (16-byte
//     chunks, L2 only) DEPTH rows ahead of use, so DRAM traffic overlaps the
//     arithmetic of the rows in flight.  Every population is read from DRAM
//     once (plus the 2 x HP halo columns and 6 warm-up rows per segment,
//     which mostly hit L2) and written once.
//   * Walls: ghost rows of phi come from loading the mirror row; a ghost mu
//     row copies its mirror row when that row exists; the ghost p row is
//     extrapolated from the two rows inside (same rules as k_step).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap_any(int x, int nx) {
    if (x < 0) x += nx;
    else if (x >= nx) x -= nx;
    if ((unsigned)x >= (unsigned)nx) {
        x %= nx;
        if (x < 0) x += nx;
    }
    return x;
}

// Shared-memory row buffers of the populations, per storage type.
template <class ST>
struct StripRow;

template <class T>
struct StripRow<PlainStore<T>> {
    using C = T;
    static constexpr int HP = 4;               // halo columns loaded each side
    static constexpr int CE = 16 / sizeof(T);  // elements per 16-byte chunk
    template <int LW>
    static constexpr size_t bytes() { return (size_t)18 * LW * sizeof(T); }
    // Issue the async copy of global row `srow`, columns x_start .. x_start+LW-1
    // (wrapped periodically), of all 18 slots into sbuf.
    template <int LW>
    __device__ __forceinline__ static void issue(char *sbuf, const char *lvl, long long NS,
                                                 long long rowbase, int x_start, int nx, int tid,
                                                 int nthr) {
        constexpr int CPS = LW / CE;  // chunks per slot
        const T *g = reinterpret_cast<const T *>(lvl);
        T *s = reinterpret_cast<T *>(sbuf);
        for (int j = tid; j < 18 * CPS; j += nthr) {
            const int sl = j / CPS, c = j - sl * CPS;
            const int xw = wrap_any(x_start + c * CE, nx);
            cp_async16(s + sl * LW + c * CE, g + sl * NS + rowbase + xw);
        }
    }
    template <int LW>
    __device__ __forceinline__ static void read_f(const char *sbuf, int c, C f[9]) {
        const T *s = reinterpret_cast<const T *>(sbuf);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = s[i * LW + c];
    }
    template <int LW>
    __device__ __forceinline__ static void read_g(const char *sbuf, int c, C g[9]) {
        const T *s = reinterpret_cast<const T *>(sbuf);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = s[(9 + i) * LW + c];
    }
};

template <class H>
struct StripRow<Store16<H>> {
    using C = float;
    using E = HalfStore<H>;
    static constexpr int HP = 8;  // 8 halves per 16-byte chunk
    template <int LW>
    static constexpr size_t bytes() { return (size_t)LW * 4 + (size_t)17 * LW * 2; }
    template <int LW>
    __device__ __forceinline__ static void issue(char *sbuf, const char *lvl, long long NS,
                                                 long long rowbase, int x_start, int nx, int tid,
                                                 int nthr) {
        constexpr int C0 = LW / 4, CH = LW / 8;  // chunks: g0 (floats), each half slot
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl + NS * 4);
        float *s0 = reinterpret_cast<float *>(sbuf);
        unsigned short *sh = reinterpret_cast<unsigned short *>(sbuf + (size_t)LW * 4);
        for (int j = tid; j < C0 + 17 * CH; j += nthr) {
            if (j < C0) {
                const int xw = wrap_any(x_start + j * 4, nx);
                cp_async16(s0 + j * 4, g0 + rowbase + xw);
            } else {
                const int jj = j - C0;
                const int sl = jj / CH, c = jj - sl * CH;
                const int xw = wrap_any(x_start + c * 8, nx);
                cp_async16(sh + sl * LW + c * 8, h + sl * NS + rowbase + xw);
            }
        }
    }
    template <int LW>
    __device__ __forceinline__ static void read_f(const char *sbuf, int c, C f[9]) {
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(sbuf + (size_t)LW * 4);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = E::dec(sh[i * LW + c]);
    }
    template <int LW>
    __device__ __forceinline__ static void read_g(const char *sbuf, int c, C g[9]) {
        const float *s0 = reinterpret_cast<const float *>(sbuf);
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(sbuf + (size_t)LW * 4);
        g[0] = s0[c];
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = E::dec(sh[(8 + i) * LW + c]);
    }
};

// Shared-memory layout of one strip CTA.
template <class T, class ST, int SW, int DEPTH>
struct StripSmem {
    using SR = StripRow<ST>;
    static constexpr int HP = SR::HP;
    static constexpr int LW = SW + 2 * HP;     // population row width
    static constexpr int NB = DEPTH + 4;       // population row buffers
    static constexpr int RPHI = 5, RMU = 4, RP = 3, RU = 2;
    static constexpr int WPHI = SW + 6, WMU = SW + 4, WQ = SW + 2;
    static constexpr size_t popb = SR::template bytes<LW>();
    static constexpr size_t pop_bytes = ((popb + 15) / 16 * 16) * NB;
    // fields: phi ring, mu ring, p ring, ps/jx/jy (1 row), and a 2-row ring
    // of ux, uy, Fx, Fy, lap mu, grad phi (x, y)
    static constexpr size_t fld_elems =
        (size_t)RPHI * WPHI + (size_t)RMU * WMU + (size_t)RP * WQ + 3 * (size_t)WQ + 7 * RU * (size_t)WQ;
    static constexpr size_t bytes = pop_bytes + fld_elems * sizeof(T);

    char *pop;
    T *phi, *mu, *p, *ps, *jx, *jy, *ux, *uy, *Fx, *Fy, *lmu, *gpx_, *gpy_;
    __device__ __forceinline__ StripSmem(char *base) {
        pop = base;
        phi = reinterpret_cast<T *>(base + pop_bytes);
        mu = phi + RPHI * WPHI;
        p = mu + RMU * WMU;
        ps = p + RP * WQ;
        jx = ps + WQ;
        jy = jx + WQ;
        ux = jy + WQ;
        uy = ux + RU * WQ;
        Fx = uy + RU * WQ;
        Fy = Fx + RU * WQ;
        lmu = Fy + RU * WQ;
        gpx_ = lmu + RU * WQ;   // grad phi, x
        gpy_ = gpx_ + RU * WQ;  // grad phi, y
    }
    __device__ __forceinline__ char *buf(int row) const {
        return pop + (size_t)((row + 64) % NB) * ((popb + 15) / 16 * 16);
    }
    // ring row pointers; column index relative to the strip's first column
    __device__ __forceinline__ T *phir(int row) const { return phi + ((row + 64) % RPHI) * WPHI + 3; }
    __device__ __forceinline__ T *mur(int row) const { return mu + ((row + 64) % RMU) * WMU + 2; }
    __device__ __forceinline__ T *pr(int row) const { return p + ((row + 64) % RP) * WQ + 1; }
    __device__ __forceinline__ int ur(int row) const { return ((row + 64) % RU) * WQ + 1; }
};

template <class T, class ST, int SW, int DEPTH>
__global__ void __launch_bounds__(SW)
k_strip(const char *__restrict__ src, char *__restrict__ dst, const KP<T> P, int seg_h) {
    using SM = StripSmem<T, ST, SW, DEPTH>;
    using SR = typename SM::SR;
    constexpr int LW = SM::LW, HP = SM::HP;
    extern __shared__ __align__(16) char smem_raw[];
    const SM s(smem_raw);
    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny, wall = P.wall;
    const long long NS = P.NS;
    const int x0 = blockIdx.x * SW;
    const int ys = blockIdx.y * seg_h;
    const int ye = min(ys + seg_h, ny);
    const int yfirst = ys - 6;
    const int xs = x0 - HP;  // first loaded column

    auto issue_row = [&](int row) {
        if (row <= ye + 2) {
            const long long rb = (long long)src_row(row, ny, wall) * nx;
            SR::template issue<LW>(s.buf(row), src, NS, rb, xs, nx, t, SW);
        }
        cp_async_commit();  // one group per row, possibly empty
    };
    // Prologue: rows yfirst+3 .. yfirst+3+DEPTH-1.
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) issue_row(yfirst + 3 + d);

    const T c3 = T(1.0 / 3.0), c6 = T(0.5 / 3.0);
    for (int y = yfirst; y < ye; ++y) {
        cp_async_wait<DEPTH - 1>();   // row y+3 has landed (this thread's chunks)
        __syncthreads();              // ... everyone's; and row y-1 is free
        issue_row(y + 3 + DEPTH);     // into the buffer of row y-1

        // 1. phi at row y+3, columns -3 .. SW+2
        {
            const char *b = s.buf(y + 3);
            T *ph = s.phir(y + 3);
            for (int c = t - 3; c < SW + 3; c += SW) {
                T g[9];
                SR::template read_g<LW>(b, c + HP, g);
                T a = g[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) a += g[i];
                ph[c] = a;
            }
        }
        // 2. sum f and j at row y+1, columns -1 .. SW
        {
            const char *b = s.buf(y + 1);
            for (int c = t - 1; c < SW + 1; c += SW) {
                T f[9];
                SR::template read_f<LW>(b, c + HP, f);
                T a = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) a += f[i];
                s.ps[c + 1] = a;
                s.jx[c + 1] = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                s.jy[c + 1] = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
            }
        }
        __syncthreads();

        // 3. mu at row y+2, columns -2 .. SW+1 (Eq. 5)
        {
            const int r = y + 2;
            T *mo = s.mur(r);
            const bool ghost = wall && (r < 0 || r >= ny);
            if (!ghost) {
                const T *pu = s.phir(r + 1), *pc = s.phir(r), *pd = s.phir(r - 1);
                T *mlow = (wall && r == 0) ? s.mur(-1) : nullptr;
                for (int c = t - 2; c < SW + 2; c += SW) {
                    const T C = pc[c];
                    const T ax = (pc[c + 1] - C) + (pc[c - 1] - C) + (pu[c] - C) + (pd[c] - C);
                    const T dg = (pu[c + 1] - C) + (pu[c - 1] - C) + (pd[c - 1] - C) + (pd[c + 1] - C);
                    const T lap = T(6) * (ax * T(1.0 / 9.0) + dg * T(1.0 / 36.0));
                    const T m = P.beta4 * (C - P.phiA) * (C - P.phiB) * (C - P.phibar) - P.kappa * lap;
                    mo[c] = m;
                    if (mlow) mlow[c] = m;  // ghost row -1 mirrors row 0
                }
            } else if (r >= ny) {
                const T *mm = s.mur(2 * ny - 1 - r);  // mirror row (already computed)
                for (int c = t - 2; c < SW + 2; c += SW) mo[c] = mm[c];
            }
            // r < 0 at a wall: row -1 is written when row 0 is computed;
            // rows below are never read.
        }
        __syncthreads();

        // 4. u, p, F, lap mu, grad phi at row y+1, columns -1 .. SW
        {
            const int r = y + 1;
            T *po = s.pr(r);
            const int uo = s.ur(r);
            if (!wall || (r >= 0 && r < ny)) {
                const T *pu = s.phir(r + 1), *pc = s.phir(r), *pd = s.phir(r - 1);
                const T *mu_ = s.mur(r + 1), *mc = s.mur(r), *md = s.mur(r - 1);
                for (int c = t - 1; c < SW + 1; c += SW) {
                    const T phi = pc[c];
                    const T gphx = T(3) * ((pc[c + 1] - pc[c - 1]) * T(1.0 / 9.0) +
                                           ((pu[c + 1] - pu[c - 1]) + (pd[c + 1] - pd[c - 1])) * T(1.0 / 36.0));
                    const T gphy = T(3) * ((pu[c] - pd[c]) * T(1.0 / 9.0) +
                                           ((pu[c + 1] + pu[c - 1]) - (pd[c - 1] + pd[c + 1])) * T(1.0 / 36.0));
                    const T M = mc[c];
                    const T gmx = T(3) * ((mc[c + 1] - mc[c - 1]) * T(1.0 / 9.0) +
                                          ((mu_[c + 1] - mu_[c - 1]) + (md[c + 1] - md[c - 1])) * T(1.0 / 36.0));
                    const T gmy = T(3) * ((mu_[c] - md[c]) * T(1.0 / 9.0) +
                                          ((mu_[c + 1] + mu_[c - 1]) - (md[c - 1] + md[c + 1])) * T(1.0 / 36.0));
                    const T ax = (mc[c + 1] - M) + (mc[c - 1] - M) + (mu_[c] - M) + (md[c] - M);
                    const T dg = (mu_[c + 1] - M) + (mu_[c - 1] - M) + (md[c - 1] - M) + (md[c + 1] - M);
                    const T lm = T(6) * (ax * T(1.0 / 9.0) + dg * T(1.0 / 36.0));
                    const T rho = P.rhoB + (phi - P.phiB) * P.drho;
                    const T Fx = -phi * gmx;
                    const T Fy = -phi * gmy - (rho - P.rhoref) * P.grav;
                    const T irc = T(3) / rho;
                    const T ux = (s.jx[c + 1] + c6 * Fx) * irc;
                    const T uy = (s.jy[c + 1] + c6 * Fy) * irc;
                    const T udr = (ux * gphx + uy * gphy) * P.drho;
                    po[c] = s.ps[c + 1] + c6 * (udr - P.gl * rho * lm);
                    s.ux[uo + c] = ux;
                    s.uy[uo + c] = uy;
                    s.Fx[uo + c] = Fx;
                    s.Fy[uo + c] = Fy;
                    s.lmu[uo + c] = lm;
                    s.gpx_[uo + c] = gphx;
                    s.gpy_[uo + c] = gphy;
                }
            } else if (r == ny) {
                // ghost row above the top wall: linear extrapolation of p
                const T *p1 = s.pr(ny - 1), *p2 = s.pr(ny - 2);
                for (int c = t - 1; c < SW + 1; c += SW) po[c] = T(2) * p1[c] - p2[c];
            }
        }
        __syncthreads();

        // 5. collide row y and push (Eqs. 22-29, Gamma_i = 1 + s_i)
        if (y >= ys) {
            const int c = t;
            const int gx = x0 + c;
            if (gx < nx) {
                const int uo = s.ur(y);
                const T *pc = s.pr(y), *pu = s.pr(y + 1);
                const T *pd = s.pr(y - 1);
                const bool lowghost = wall && y == 0;
                T pdm = lowghost ? T(2) * pc[c - 1] - pu[c - 1] : pd[c - 1];
                T pd0 = lowghost ? T(2) * pc[c] - pu[c] : pd[c];
                T pdp = lowghost ? T(2) * pc[c + 1] - pu[c + 1] : pd[c + 1];
                const T gpx = T(3) * ((pc[c + 1] - pc[c - 1]) * T(1.0 / 9.0) +
                                      ((pu[c + 1] - pu[c - 1]) + (pdp - pdm)) * T(1.0 / 36.0));
                const T gpy = T(3) * ((pu[c] - pd0) * T(1.0 / 9.0) +
                                      ((pu[c + 1] + pu[c - 1]) - (pdm + pdp)) * T(1.0 / 36.0));
                const T phi = s.phir(y)[c];
                const T mu = s.mur(y)[c];
                const T pv = pc[c];
                const T ux = s.ux[uo + c], uy = s.uy[uo + c];
                const T Fx = s.Fx[uo + c], Fy = s.Fy[uo + c];
                const T lm = s.lmu[uo + c];
                const T rho = P.rhoB + (phi - P.phiB) * P.drho;
                const T grx = P.drho * s.gpx_[uo + c], gry = P.drho * s.gpy_[uo + c];
                T f[9], g[9];
                const char *b = s.buf(y);
                SR::template read_f<LW>(b, c + HP, f);
                SR::template read_g<LW>(b, c + HP, g);

                const T uu = ux * ux + uy * uy;
                const T amu = P.alpha * mu;
                const T srcF = c3 * rho * P.gl * lm;
                const T gq = -T(3) * phi / rho;
                const T dx = gpx - Fx, dy = gpy - Fy;
                const T uF = ux * Fx + uy * Fy, uR = ux * grx + uy * gry, uD = ux * dx + uy * dy;
                const T rho3 = c3 * rho;
                T fv[9], gv[9];
                int sl[9];
                long long kk[9];
                const long long k = (long long)y * nx + gx;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
                    const T w = T(D2Q9::w(i));
                    const T cu = T(cx) * ux + T(cy) * uy;
                    const T si = cu * (T(3) + T(4.5) * cu) - T(1.5) * uu;
                    const T eF = (T(cx) * Fx + T(cy) * Fy) - uF;
                    const T eR = (T(cx) * grx + T(cy) * gry) - uR;
                    const T eD = (T(cx) * dx + T(cy) * dy) - uD;
                    const T G1 = T(1) + si;
                    const T Fi = w * (G1 * eF + (si * c3) * eR - srcF);
                    const T Gi = w * gq * G1 * eD;
                    const T feq = w * (pv + rho3 * si);
                    const T H = (i == 0) ? phi - T(1.0 - D2Q9::w(0)) * amu : w * amu;
                    const T geq = H + w * phi * si;
                    T fs = f[i] - (f[i] - feq) * P.itf + P.pf * Fi;
                    T gs = g[i] - (g[i] - geq) * P.itg + P.pg * Gi;
                    const int yd = y + cy;
                    if (wall && (yd < 0 || yd >= ny)) {
                        const T cuw = T(cx) * (yd < 0 ? P.uwb : P.uwt);
                        fs -= T(2) * w * rho * cuw;
                        gs -= T(6) * w * phi * cuw;
                        sl[i] = D2Q9::opp(i);
                        kk[i] = k;
                    } else {
                        int xd = gx + cx;
                        xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                        const int yy = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
                        sl[i] = i;
                        kk[i] = (long long)yy * nx + xd;
                    }
                    fv[i] = fs;
                    gv[i] = gs;
                }
                ST::store(dst, NS, sl, kk, fv, gv, phi);
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace lbm
