// lbm_strip_lag.cuh — the strip form of the lagged-grad-p variant.
//
// The variant (not the paper's scheme; a measurement of what the synchrony
// of Sec. 3 costs): G_i of Eq. 29 takes grad p from the pressure of the
// previous step, which each level stores beside its populations (one slot
// P of NS elements of the field type, after the population slots).  Before
// the first step P holds the initial state's p = 0.
//
// The step then reaches 2 cells instead of 3 (p <- lap mu <- lap phi), and
// p, u, F, lap mu and grad phi of a cell are needed by that cell only, so
// the strip pipeline is one stage shorter than k_strip's: iteration y
//   1. phi at row y+2 from the g row (columns -2 .. SW+1),
//   3. mu at row y+1 (columns -1 .. SW),
//   4. Sigma f, j of row y, then grad phi, grad mu, lap mu, F, u (Eq. 31) and
//      p (Eq. 32) of the thread's own column, grad P from the stored
//      previous-step rows y-1 .. y+1, the collision of row y and the push;
//      p goes to the P slot of the other level.
// Three barriers per row (k_strip: four), 4 warm-up rows per segment (6),
// and no step that needs a halo pass of the heavy work.  The halo of P is
// one 16-byte chunk per side; ghost rows of P at walls are extrapolated as
// in the synchronous step.
#pragma once

#include "lbm_strip.cuh"

namespace lbm {

// Shared-memory layout of one lagged-strip CTA.
template <class T, class ST, int SW, int DEPTH>
struct LagSmem {
    using SR = StripRow<ST, SW>;
    using C = typename SR::C;  // field type: T for plain storage, float for 16-bit
    static constexpr int HP = SR::HP;
    static constexpr int LW = SR::LW;
    // g rows: phi at y+2, collision at y; f rows: row y only; P rows y-1..y+1
    static constexpr int NBG = DEPTH + 3, NBF = DEPTH + 1, NBP = DEPTH + 3;
    static constexpr int CEP = 16 / (int)sizeof(C);  // P elements per 16-byte chunk
    static constexpr int LWP = SW + 2 * CEP;          // P row: one chunk of halo per side
    static constexpr int CHP = LWP / CEP;             // chunks per P row
    // field rings: phi rows y-1..y+2, mu rows y-1..y+1
    static constexpr int RPHI = 4, RMU = 3;
    static constexpr int WPHI = SW + 4, WMU = SW + 2;
    static constexpr int ET = (int)sizeof(T);
    static constexpr size_t gb = (SR::gbytes + 15) / 16 * 16;
    static constexpr size_t fb = (SR::fbytes + 15) / 16 * 16;
    static constexpr size_t pb = (size_t)LWP * sizeof(C);
    static constexpr size_t pop_bytes = gb * NBG + fb * NBF + pb * NBP;
    static constexpr size_t bytes = pop_bytes + sizeof(T) * ((size_t)RPHI * WPHI + (size_t)RMU * WMU);
    static_assert(CHP <= strip_threads(SW), "one P chunk per thread");
    // tensor-tile staging of the g and f rows (FP32), as in StripSmem: the
    // rows issued in one iteration complete on one of DEPTH + 1 mbarriers
    // after the rings; row buffers on 128-byte boundaries
    static constexpr int NBAR = DEPTH + 1;
    static constexpr size_t bar_off = (bytes + 7) / 8 * 8;
    static constexpr size_t bytes_tma = bar_off + 8 * (size_t)NBAR;
    static constexpr bool TMA_ROWS = gb % 128 == 0 && fb % 128 == 0;
};

// Ring slots (byte offsets into shared memory) of the rows live at
// iteration y: g[k], f[k] hold row y+k; p[k], ph[k], mu[k] row y-1+k.
template <class LS>
struct LagRings {
    int g[LS::NBG], f[LS::NBF], p[LS::NBP], ph[LS::RPHI], mu[LS::RMU];
    __device__ __forceinline__ LagRings() {
        constexpr int ET = LS::ET;
        constexpr int b_f = (int)(LS::gb * LS::NBG);
        constexpr int b_p = b_f + (int)(LS::fb * LS::NBF);
        constexpr int b_ph = (int)LS::pop_bytes;
        constexpr int b_mu = b_ph + LS::RPHI * LS::WPHI * ET;
#pragma unroll
        for (int k = 0; k < LS::NBG; ++k) g[k] = k * (int)LS::gb;
#pragma unroll
        for (int k = 0; k < LS::NBF; ++k) f[k] = b_f + k * (int)LS::fb;
#pragma unroll
        for (int k = 0; k < LS::NBP; ++k) p[k] = b_p + k * (int)LS::pb;
#pragma unroll
        for (int k = 0; k < LS::RPHI; ++k) ph[k] = b_ph + (k * LS::WPHI + 2) * ET;
#pragma unroll
        for (int k = 0; k < LS::RMU; ++k) mu[k] = b_mu + (k * LS::WMU + 1) * ET;
    }
    template <int N>
    __device__ __forceinline__ static void rot(int (&a)[N]) {
        const int t = a[0];
#pragma unroll
        for (int k = 0; k + 1 < N; ++k) a[k] = a[k + 1];
        a[N - 1] = t;
    }
    __device__ __forceinline__ void advance() {
        rot(g);
        rot(f);
        rot(p);
        rot(ph);
        rot(mu);
    }
};

// Push of one collided cell through the general path (periodic wrap in x
// and y, halfway bounce-back with the moving-wall term at y walls).
template <class T, class ST>
__device__ __forceinline__ void push_general(char *dst, const KP<T> &P, T fv[9], T gv[9], T phi,
                                             T rho, int gx, int y) {
    const int nx = P.nx, ny = P.ny;
    int sl[9];
    long long kk[9];
    const long long k = (long long)y * nx + gx;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
        const int yd = y + cy;
        if (P.wall && (yd < 0 || yd >= ny)) {
            const T w = T(D2Q9::w(i));
            const T cuw = T(cx) * (yd < 0 ? P.uwb : P.uwt);
            fv[i] -= T(2) * w * rho * cuw;
            gv[i] -= T(6) * w * phi * cuw;
            sl[i] = D2Q9::opp(i);
            kk[i] = k;
        } else {
            int xd = gx + cx;
            xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
            const int yy = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
            sl[i] = i;
            kk[i] = (long long)yy * nx + xd;
        }
    }
    ST::store(dst, P.NS, sl, kk, fv, gv, phi);
}

// One work item: columns x0 .. x0+SW-1, rows ys .. ye-1.  `poff` is the
// byte offset of the P slot within a level.  TMA: `map` is the source
// level's 3-D tensor map; strips whose rows do not wrap in x take their g
// and f rows from it (the P rows stay 16-byte chunk copies).
template <class T, class ST, int SW, int DEPTH, bool TMA = false>
__device__ __forceinline__ void strip_body_lag(const char *__restrict__ src, char *__restrict__ dst,
                                               const KP<T> &P, long long poff, const int x0,
                                               const int ys, const int ye, char *smem_raw,
                                               const CUtensorMap *map = nullptr) {
    using LS = LagSmem<T, ST, SW, DEPTH>;
    using SR = typename LS::SR;
    using C = typename LS::C;
    constexpr int HP = LS::HP;
    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny, wall = P.wall;
    const int NS = (int)P.NS;
    const int yfirst = ys - 4;

    typename SR::Desc desc;
    const int active = nx - x0 < SW ? nx - x0 : SW;
    SR::describe(desc, t, P.NS, x0 - HP, nx, active + 2 * HP);
    // P row chunk of this thread (one 16-byte chunk, columns x0-CEP .. )
    int pgo = -1;
    if (t < LS::CHP && t * LS::CEP < active + 2 * LS::CEP)
        pgo = wrap_any(x0 - LS::CEP + t * LS::CEP, nx);
    const bool tma = TMA && x0 - HP >= 0 && x0 - HP + SR::LW <= nx;
    unsigned bars = 0;
    if constexpr (TMA) {
        static_assert(LS::TMA_ROWS, "TMA rows need 128-byte aligned row buffers");
        bars = smem_u32(smem_raw + LS::bar_off);
        if (tma && t == 0) {
            for (int k = 0; k < LS::NBAR; ++k) mbar_init(bars + 8 * k, 1);
            mbar_init_fence();
        }
    }
    __syncthreads();

    LagRings<LS> R;
    auto at = [&](int off) { return smem_raw + off; };
    auto atT = [&](int off) { return reinterpret_cast<T *>(smem_raw + off); };
    auto atC = [&](int off) { return reinterpret_cast<C *>(smem_raw + off); };
    const C *Psrc = reinterpret_cast<const C *>(src + poff);
    C *Pdst = reinterpret_cast<C *>(dst + poff);

    // Barrier and phase parity of the rows issued for iteration it (the
    // NBAR barriers in turn from yfirst on, each once every NBAR
    // iterations).
    auto ibar = [&](int it) { return bars + 8u * (unsigned)((it - yfirst) % LS::NBAR); };
    auto ipar = [&](int it) { return (unsigned)((it - yfirst) / LS::NBAR) & 1u; };
    // Iteration y reads g row y+2, f row y and P row y+1 first; all are
    // issued DEPTH iterations earlier, as one commit group (and, with
    // tensor tiles, the g and f rows on one mbarrier).  Every iteration of
    // the loop has its g row, so every barrier it waits on was armed.
    auto issue_for = [&](int it, int gslot, int fslot, int pslot) {
        const int gr = it + 2, fr = it, pr = it + 1;
        const bool g_in = gr <= ye + 1, f_in = fr >= ys && fr < ye;
        if (tma) {
            if (t == 0 && (g_in || f_in)) {
                constexpr unsigned row_bytes = (unsigned)(9 * SR::LW * sizeof(T));
                const unsigned bar = ibar(it);
                mbar_expect_tx(bar, (g_in ? row_bytes : 0u) + (f_in ? row_bytes : 0u) + P.tx_extra);
                if (g_in) tma_load_3d(smem_u32(at(gslot)), map, bar, x0 - HP, src_row(gr, ny, wall), 9);
                if (f_in) tma_load_3d(smem_u32(at(fslot)), map, bar, x0 - HP, src_row(fr, ny, wall), 0);
            }
        } else {
            if (g_in) SR::issue_g(desc, at(gslot), src, src_row(gr, ny, wall) * nx);
            if (f_in) SR::issue_f(desc, at(fslot), src, src_row(fr, ny, wall) * nx);
        }
        if (pr >= ys - 1 && pr <= ye && pgo >= 0)
            cp_async16(atC(pslot) + t * LS::CEP, Psrc + (src_row(pr, ny, wall) * nx + pgo));
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) issue_for(yfirst + d, R.g[d + 2], R.f[d], R.p[d + 2]);

    const bool x_inner = x0 > 0 && x0 + SW < nx;
    const T c6 = T(0.5 / 3.0);

    for (int y = yfirst; y < ye; ++y) {
        cp_async_wait<DEPTH - 1>();  // this thread's P chunk of row y+1
        if (tma) {
            // g row y+2 and f row y have landed (bounded wait); the CTA
            // barrier also publishes every thread's P chunk
            if (__syncthreads_or(!mbar_wait(ibar(y), ipar(y)))) {
                if (t == 0 && P.err) atomicOr(P.err, 1u);
                // the loads of iterations y+1 .. y+DEPTH-1 are still in
                // flight into this CTA's shared memory: wait (bounded)
                for (int d = 1; d < DEPTH; ++d)
                    if (y + d < ye) mbar_wait(ibar(y + d), ipar(y + d));
                cp_async_wait<0>();
                return;
            }
        } else {
            __syncthreads();
        }
        issue_for(y + DEPTH, R.g[LS::NBG - 1], R.f[LS::NBF - 1], R.p[LS::NBP - 1]);

        // 1. phi at row y+2, columns -2 .. SW+1
        {
            const char *b = at(R.g[2]);
            T *ph = atT(R.ph[3]);
            columns<SW, 2, 3>(t, [&](int c) {
                C g[9];
                SR::read_g(b, c + HP, g);
                ph[c] = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
            });
        }
        __syncthreads();

        // 3. mu at row y+1, columns -1 .. SW (Eq. 5)
        {
            const int r = y + 1;
            T *mo = atT(R.mu[2]);
            const bool ghost = wall && (r < 0 || r >= ny);
            if (!ghost) {
                const T *pu = atT(R.ph[3]), *pc = atT(R.ph[2]), *pd = atT(R.ph[1]);
                T *mlow = (wall && r == 0) ? atT(R.mu[1]) : nullptr;  // row -1
                columns<SW, 1, 1>(t, [&](int c) {
                    const T Cc = pc[c];
                    const T ax = ((pc[c + 1] - Cc) + (pc[c - 1] - Cc)) + ((pu[c] - Cc) + (pd[c] - Cc));
                    const T dg = ((pu[c + 1] - Cc) + (pu[c - 1] - Cc)) + ((pd[c - 1] - Cc) + (pd[c + 1] - Cc));
                    const T lap = T(2.0 / 3.0) * ax + T(1.0 / 6.0) * dg;
                    const T m = P.beta4 * (Cc - P.phiA) * (Cc - P.phiB) * (Cc - P.phibar) - P.kappa * lap;
                    mo[c] = m;
                    if (mlow) mlow[c] = m;
                });
            } else if (r == ny) {
                const T *mm = atT(R.mu[1]);  // mirror row ny-1
                columns<SW, 1, 1>(t, [&](int c) { mo[c] = mm[c]; });
            }
        }
        __syncthreads();

        // 4. row y, own column: moments, gradients, u, p, grad P, collision
        if (y >= ys) {
            const int c = t;
            const int gx = x0 + c;
            if (c < SW && gx < nx) {
                const T *pu = atT(R.ph[2]), *pc = atT(R.ph[1]), *pd = atT(R.ph[0]);
                const T *mu_ = atT(R.mu[2]), *mc = atT(R.mu[1]), *md = atT(R.mu[0]);
                C f[9], g[9];
                SR::read_f(at(R.f[0]), c + HP, f);
                const T sf = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
                const T jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                const T jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
                const T phi = pc[c];
                const T pul = pu[c - 1], pur = pu[c + 1], pdl = pd[c - 1], pdr = pd[c + 1];
                const T gphx = T(1.0 / 3.0) * (pc[c + 1] - pc[c - 1]) + T(1.0 / 12.0) * ((pur - pul) + (pdr - pdl));
                const T gphy = T(1.0 / 3.0) * (pu[c] - pd[c]) + T(1.0 / 12.0) * ((pur + pul) - (pdl + pdr));
                const T M = mc[c];
                const T mul = mu_[c - 1], mur = mu_[c + 1], mdl = md[c - 1], mdr = md[c + 1];
                const T mcl = mc[c - 1], mcr = mc[c + 1], mcu = mu_[c], mcd = md[c];
                const T gmx = T(1.0 / 3.0) * (mcr - mcl) + T(1.0 / 12.0) * ((mur - mul) + (mdr - mdl));
                const T gmy = T(1.0 / 3.0) * (mcu - mcd) + T(1.0 / 12.0) * ((mur + mul) - (mdl + mdr));
                const T lm = T(2.0 / 3.0) * (((mcl - M) + (mcr - M)) + ((mcu - M) + (mcd - M))) +
                             T(1.0 / 6.0) * (((mur - M) + (mul - M)) + ((mdl - M) + (mdr - M)));
                const T rho = P.rhoB + (phi - P.phiB) * P.drho;
                const T Fx = -phi * gmx;
                const T Fy = -phi * gmy - (rho - P.rhoref) * P.grav;
                const T irc = T(3) * rcp_fast(rho);
                const T ux = (jx + c6 * Fx) * irc;
                const T uy = (jy + c6 * Fy) * irc;
                const T pv = sf + c6 * ((ux * gphx + uy * gphy) * P.drho - P.gl * rho * lm);
                // grad of the previous step's p; ghost rows at walls extrapolated
                const C *qc = atC(R.p[1]) + LS::CEP + c, *qu = atC(R.p[2]) + LS::CEP + c,
                        *qd = atC(R.p[0]) + LS::CEP + c;
                const bool lowghost = wall && y == 0, highghost = wall && y == ny - 1;
                const T qcm = qc[-1], qcp = qc[1];
                T qum = qu[-1], qu0 = qu[0], qup = qu[1];
                T qdm = qd[-1], qd0 = qd[0], qdp = qd[1];
                if (lowghost) {
                    qdm = T(2) * qcm - qum;
                    qd0 = T(2) * qc[0] - qu0;
                    qdp = T(2) * qcp - qup;
                }
                if (highghost) {
                    qum = T(2) * qcm - qdm;
                    qu0 = T(2) * qc[0] - qd0;
                    qup = T(2) * qcp - qdp;
                }
                const T gpx = T(1.0 / 3.0) * (qcp - qcm) + T(1.0 / 12.0) * ((qup - qum) + (qdp - qdm));
                const T gpy = T(1.0 / 3.0) * (qu0 - qd0) + T(1.0 / 12.0) * ((qup + qum) - (qdm + qdp));
                SR::read_g(at(R.g[0]), c + HP, g);
                T fv[9], gv[9];
                collide(P, CellState<T>{phi, M, pv, rho, ux, uy, Fx, Fy, lm, gphx, gphy, gpx, gpy},
                        f, g, fv, gv);
                Pdst[(long long)y * nx + gx] = C(pv);
                if (x_inner && y > 0 && y < ny - 1)
                    SR::store_fast(dst, NS, nx, y * nx + gx, fv, gv, phi);
                else
                    push_general<T, ST>(dst, P, fv, gv, phi, rho, gx, y);
            }
        }
        R.advance();
    }
    cp_async_wait<0>();
}

template <class T, class ST, int SW, int DEPTH>
__global__ void __launch_bounds__(strip_threads(SW))
k_strip_lag(const char *__restrict__ src, char *__restrict__ dst, const __grid_constant__ KP<T> P,
            long long poff, int seg_h) {
    extern __shared__ __align__(16) char smem_raw[];
    const int ys = blockIdx.y * seg_h;
    strip_body_lag<T, ST, SW, DEPTH>(src, dst, P, poff, blockIdx.x * SW, ys,
                                     min(ys + seg_h, P.ny), smem_raw);
}

// The same with tensor-tile staging of the g and f rows (FP32): `map`
// describes the source level (x, row, slot).
template <class T, class ST, int SW, int DEPTH>
__global__ void __launch_bounds__(strip_threads(SW))
k_strip_lag_tma(const char *__restrict__ src, char *__restrict__ dst, const __grid_constant__ KP<T> P,
                long long poff, int seg_h, const __grid_constant__ CUtensorMap map) {
    extern __shared__ __align__(128) char smem_raw[];
    const int ys = blockIdx.y * seg_h;
    strip_body_lag<T, ST, SW, DEPTH, true>(src, dst, P, poff, blockIdx.x * SW, ys,
                                           min(ys + seg_h, P.ny), smem_raw, &map);
}

}  // namespace lbm
