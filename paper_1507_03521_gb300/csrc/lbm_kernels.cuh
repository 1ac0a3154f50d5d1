// lbm_kernels.cuh — CUDA kernels of one time step of the quasi-incompressible
// phase-field lattice Boltzmann scheme (Yang & Guo, arXiv 1507.03521), D2Q9,
// for sm_103a.  Included by one translation unit per storage type.
//
// Naming follows the paper: f_i is the flow population (Eq. 22, tau_f),
// g_i the phase-field population (Eq. 23, tau_g).
//
// Design of the step (one kernel launch per time step):
//   * Populations live in two time levels (ping-pong), structure of arrays:
//     slot s of cell k at s * NS + k (NS = padded cell count).  A level
//     holds the post-streaming populations of its time, so every load of
//     a cell's own populations is local and coalesced.
//   * A CTA owns a 32 x TY tile.  It rebuilds the moments it needs on a
//     halo instead of reading moment arrays: phi = sum g_i on a 3-cell halo
//     (grad p needs p on a 1-ring, p needs lap mu, mu needs lap phi),
//     sum f_i and sum c_i f_i on a 1-cell halo.  Halo loads of the
//     neighbouring tiles' populations are served by L2; each population is
//     read once and written once from DRAM per step.
//   * mu (Eq. 5), then u (Eq. 31) and p (Eq. 32) are built in shared memory
//     on shrinking rings; each owned cell then forms grad p, collides both
//     populations (Eqs. 22-29) from registers and pushes the results to
//     their destination cells of the other level (left-hand sides of
//     Eqs. 22-23), bouncing back at walls.
//   * The same kernel in FIELDS mode writes the macroscopic fields of the
//     current level instead of colliding.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace lbm {

// D2Q9 (end of Sec. 3): c_0 = 0, c_1..4 axis-aligned at angles (i-1) pi/2,
// c_5..8 diagonal at angles (2i-1) pi/4; w = 4/9, 1/9, 1/36; cs2 = 1/3.
struct D2Q9 {
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};
static_assert(D2Q9::opp(1) == 3 && D2Q9::opp(2) == 4 && D2Q9::opp(3) == 1 && D2Q9::opp(4) == 2,
              "opposite of axis directions");
static_assert(D2Q9::opp(5) == 7 && D2Q9::opp(6) == 8 && D2Q9::opp(7) == 5 && D2Q9::opp(8) == 6,
              "opposite of diagonal directions");

// MODE_ADJC: the reverse step's first kernel: per cell, the forward fields
// that the adjoint of the step linearises about and the later reverse
// kernels read, then the streaming and collision adjoint about them
// (AdjCell, lbm_adjoint.cuh).
enum { MODE_STEP = 0, MODE_FIELDS = 1, MODE_ADJC = 3 };

// Kernel parameters, converted once to the compute type T on the host.
template <class T>
struct KP {
    int nx, ny, wall;
    long long NS;           // slot stride (padded cell count)
    // Rows held and stepped (strip kernel).  The whole domain: slab = 0,
    // y0 = 0, rows = ny, ya..yb = 0..ny.  A y-slab of a decomposed domain:
    // slab = 1, the level holds global rows y0 .. y0+rows-1 (its own rows
    // ya..yb-1 and 3 ghost rows on each side), with no wrap in y.
    int slab, y0, rows, ya, yb;
    T phiA, phiB, phibar;   // bulk order parameters and their mean
    T rhoB, drho;           // rho = rhoB + (phi - phiB) drho (Eq. 11)
    T kappa, beta4, beta;   // kappa, 4 beta, beta
    T alpha, gl;            // alpha; gamma * lambda
    T grav, rhoref;         // F_b,y = -(rho - rhoref) grav
    T itf, itg, pf, pg;     // 1/tau_f, 1/tau_g, 1 - 1/(2 tau_f), 1 - 1/(2 tau_g)
    T uwb, uwt;             // wall x-velocities (bottom, top)
    unsigned *err;          // error word: bit 0 set when a bounded wait ran out (may be null)
    unsigned tx_extra;      // test hook: bytes a tile load announces beyond what it brings (0)
#ifdef LBM_DEBUG
    unsigned *dbg;          // bounds-check error word (LBM_DEBUG builds)
#endif
};

// Index checks of the LBM_DEBUG build.  LBM_IDX_OK(P, cond, code) is true
// in release builds; in a LBM_DEBUG build a false `cond` sets bit `code` of
// the handle's error word (which the next synchronising call reports as
// LBM_ERR_STATE) and the caller skips the access.  Codes: 1 population row
// copied to shared memory, 2 population stored, 3 shared row column read,
// 4 field-ring column, 5 population loaded by the tile kernel.
#ifdef LBM_DEBUG
__device__ __forceinline__ bool dbg_ok(unsigned *w, bool ok, unsigned code) {
    if (!ok && w) atomicOr(w, 1u << code);
    return ok;
}
#define LBM_IDX_OK(P, cond, code) ::lbm::dbg_ok((P).dbg, (cond), (code))
#else
#define LBM_IDX_OK(P, cond, code) true
#endif

// Output pointers of FIELDS mode (any may be null).
template <class T>
struct FieldOut {
    T *phi, *rho, *p, *ux, *uy, *mu, *P;
    // MODE_ADJC: base of the adjoint's field arrays (AdjArr), their stride,
    // and 4 beta and kappa per unit sigma (for mu per unit sigma)
    T *adj = nullptr;
    long long adj_ns = 0;
    T beta1x4 = T(0), kappa1 = T(0);
    // MODE_ADJC: lambda_{t+1} (read) and lambda_t (written)
    const T *lam_next = nullptr;
    T *lam = nullptr;
};

template <class T>
struct AdjCell;  // MODE_ADJC's per-cell work, defined in lbm_adjoint.cuh

// ------------------------------------------------------------ storage

// FP64 / FP32: all 18 populations in the compute type.
// Level layout: f_0..f_8 then g_0..g_8, each NS elements.
template <class T>
struct PlainStore {
    using C = T;
    static constexpr size_t level_bytes_per_cell = 18 * sizeof(T);
    static size_t level_bytes(long long NS) { return (size_t)NS * 18 * sizeof(T); }
    // Byte offset and element size of population slot q (f_0..f_8 = 0..8,
    // g_0..g_8 = 9..17) within a level.
    static void slot_span(long long NS, int q, size_t *off, size_t *elem) {
        *off = (size_t)q * NS * sizeof(T);
        *elem = sizeof(T);
    }
    __device__ __forceinline__ static void load(const char *lvl, long long NS, long long k,
                                                C f[9], C g[9]) {
        const T *b = reinterpret_cast<const T *>(lvl);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = __ldg(b + i * NS + k);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = __ldg(b + (9 + i) * NS + k);
    }
    __device__ __forceinline__ static C load_phi(const char *lvl, long long NS, long long k) {
        const T *b = reinterpret_cast<const T *>(lvl) + 9 * NS + k;
        C s = __ldg(b);
#pragma unroll
        for (int i = 1; i < 9; ++i) s += __ldg(b + i * NS);
        return s;
    }
    // In FP32, g_0 (which stays on its cell) is stored as phi minus the
    // other eight outgoing values: the collision conserves sum_i g_i = phi
    // exactly in exact arithmetic, and this keeps it so up to one FP32
    // rounding per cell, so sum phi does not drift with the rounding of g_0.
    // FP64 stores the collision's g_0 as computed.
    __device__ __forceinline__ static C g0_value(const C gv[9], C phi) {
        if (sizeof(T) != 4) return gv[0];
        C rest = phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) rest -= gv[i];
        return rest;
    }
    // fv/gv: final values per source direction i, written to slot sl[i] of
    // cell kk[i].  phi: the source cell's order parameter.
    __device__ __forceinline__ static void store(char *lvl, long long NS, const int sl[9],
                                                 const long long kk[9], const C fv[9],
                                                 const C gv[9], C phi) {
        T *b = reinterpret_cast<T *>(lvl);
#pragma unroll
        for (int i = 0; i < 9; ++i) b[sl[i] * NS + kk[i]] = fv[i];
        b[9 * NS + kk[0]] = g0_value(gv, phi);  // slot 0 never moves and never bounces
#pragma unroll
        for (int i = 1; i < 9; ++i) b[(9 + sl[i]) * NS + kk[i]] = gv[i];
    }
};

// 16-bit storage with FP32 arithmetic.  f_0..f_8 and g_1..g_8 are, at rest
// (u = 0, p = 0, mu = 0), equal to zero: they are stored directly as their
// deviation from the rest equilibrium, scaled by SCALE and rounded to the
// 16-bit type H.  g_0, which carries phi at rest, stays in FP32 and absorbs
// the rounding of the other eight: g_0 is stored as phi - sum_{i>0} g_i(read
// back), so sum_i g_i leaving each cell equals its phi up to one FP32
// rounding and sum phi is conserved.
// Level layout: g_0 (NS floats), then f_0..f_8 and g_1..g_8 (17 NS of H).
template <class H>
struct HalfStore;

template <>
struct HalfStore<__half> {
    static constexpr float SCALE = 1024.0f, ISCALE = 1.0f / 1024.0f;
    __device__ __forceinline__ static unsigned short enc(float v) {
        return __half_as_ushort(__float2half_rn(v * SCALE));
    }
    __device__ __forceinline__ static float dec(unsigned short h) {
        return __half2float(__ushort_as_half(h)) * ISCALE;
    }
};

template <>
struct HalfStore<__nv_bfloat16> {
    __device__ __forceinline__ static unsigned short enc(float v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    __device__ __forceinline__ static float dec(unsigned short h) {
        return __bfloat162float(__ushort_as_bfloat16(h));
    }
};

template <class H>
struct Store16 {
    using C = float;
    using E = HalfStore<H>;
    static size_t level_bytes(long long NS) { return (size_t)NS * (4 + 17 * 2); }
    // slot q (f_0..f_8 = 0..8, g_0..g_8 = 9..17): g_0 in FP32 first, then
    // the 16-bit slots f_0..f_8, g_1..g_8
    static void slot_span(long long NS, int q, size_t *off, size_t *elem) {
        if (q == 9) {
            *off = 0;
            *elem = 4;
        } else {
            *off = (size_t)NS * 4 + (size_t)(q < 9 ? q : q - 1) * NS * 2;
            *elem = 2;
        }
    }
    // slot index of f_i: i; of g_i (i >= 1): 8 + i
    __device__ __forceinline__ static void load(const char *lvl, long long NS, long long k,
                                                C f[9], C g[9]) {
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl + NS * 4);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = E::dec(__ldg(h + i * NS + k));
        g[0] = __ldg(g0 + k);
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = E::dec(__ldg(h + (8 + i) * NS + k));
    }
    __device__ __forceinline__ static C load_phi(const char *lvl, long long NS, long long k) {
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl + NS * 4);
        C s = __ldg(g0 + k);
#pragma unroll
        for (int i = 1; i < 9; ++i) s += E::dec(__ldg(h + (8 + i) * NS + k));
        return s;
    }
    __device__ __forceinline__ static void store(char *lvl, long long NS, const int sl[9],
                                                 const long long kk[9], const C fv[9],
                                                 const C gv[9], C phi) {
        float *g0 = reinterpret_cast<float *>(lvl);
        unsigned short *h = reinterpret_cast<unsigned short *>(lvl + NS * 4);
#pragma unroll
        for (int i = 0; i < 9; ++i) h[sl[i] * NS + kk[i]] = E::enc(fv[i]);
        float rest = phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            unsigned short q = E::enc(gv[i]);
            rest -= E::dec(q);
            h[(8 + sl[i]) * NS + kk[i]] = q;
        }
        g0[kk[0]] = rest;  // slot 0 never moves and never bounces
    }
};

// 16-bit storage of the deviations from the rest equilibrium, FP32
// arithmetic.  At rest (u = 0) the equilibria of Eqs. 24-27 are
//   f_i = w_i p,   g_i = w_i alpha mu (i >= 1),   g_0 = phi - (1 - w_0) alpha mu,
// so a population that arrives at cell y is stored as its deviation from
// the rest equilibrium at y's own p and alpha mu of the previous time
// level: d f_i = f_i - w_i P_y, d g_i = g_i - w_i A_y (i >= 1).  The sender
// of a population knows its destination's p and mu (they are on chip when
// it collides), and cell y stores its own P_y and A_y beside its
// populations, so encoder and decoder use the same references.  P_y and A_y
// are p and alpha mu cut to their upper 16 bits (a BF16 value rounded
// toward zero): any value serves as a reference as long as both sides use
// it, and this one costs one bit operation each way.  g_0 stays in FP32 as
// phi - sum_{i>0} g_i(decoded), as in Store16.
// Level layout: g_0 (NS floats), then 19 NS of H: f_0..f_8, g_1..g_8, then
// the reference words P (slot 17) and A (slot 18).
template <class H>
struct Store16D {
    using C = float;
    using E = HalfStore<H>;
    static constexpr bool kDev = true;
    static size_t level_bytes(long long NS) { return (size_t)NS * (4 + 19 * 2); }
    static void slot_span(long long NS, int q, size_t *off, size_t *elem) {
        Store16<H>::slot_span(NS, q, off, elem);
    }
    // reference words: the upper half of the FP32 bit pattern
    __host__ __device__ __forceinline__ static unsigned short ref_word(float v) {
#ifdef __CUDA_ARCH__
        return (unsigned short)(__float_as_uint(v) >> 16);
#else
        unsigned u;
        memcpy(&u, &v, 4);
        return (unsigned short)(u >> 16);
#endif
    }
    __device__ __forceinline__ static float ref_value(unsigned short r) {
        return __uint_as_float((unsigned)r << 16);
    }
    // p or alpha mu cut to its reference value
    __device__ __forceinline__ static float ref_cut(float v) {
        return __uint_as_float(__float_as_uint(v) & 0xffff0000u);
    }
    // decoded population: stored deviation plus w_i times the reference
    // (the same rounding at the encoder, which needs the decoded g_i)
    __device__ __forceinline__ static float rebuild(unsigned short q, float wref) {
        return __fadd_rn(E::dec(q), wref);
    }
    __device__ __forceinline__ static void load(const char *lvl, long long NS, long long k,
                                                C f[9], C g[9]) {
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl + NS * 4);
        const float Pr = ref_value(__ldg(h + 17 * NS + k)), Ar = ref_value(__ldg(h + 18 * NS + k));
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = rebuild(__ldg(h + i * NS + k), __fmul_rn(float(D2Q9::w(i)), Pr));
        g[0] = __ldg(g0 + k);
#pragma unroll
        for (int i = 1; i < 9; ++i)
            g[i] = rebuild(__ldg(h + (8 + i) * NS + k), __fmul_rn(float(D2Q9::w(i)), Ar));
    }
    __device__ __forceinline__ static C load_phi(const char *lvl, long long NS, long long k) {
        C f[9], g[9];
        load(lvl, NS, k, f, g);
        C s = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) s += g[i];
        return s;
    }
    // fv/gv: final values per source direction i, written to slot sl[i] of
    // cell kk[i], whose reference values (already cut) are rP[i], rA[i];
    // ownP, ownA: this cell's p and alpha mu (its own reference words).
    __device__ __forceinline__ static void store(char *lvl, long long NS, const int sl[9],
                                                 const long long kk[9], const C fv[9],
                                                 const C gv[9], C phi, const float rP[9],
                                                 const float rA[9], float ownP, float ownA) {
        float *g0 = reinterpret_cast<float *>(lvl);
        unsigned short *h = reinterpret_cast<unsigned short *>(lvl + NS * 4);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float wP = __fmul_rn(float(D2Q9::w(i)), rP[i]);
            h[sl[i] * NS + kk[i]] = E::enc(__fsub_rn(fv[i], wP));
        }
        float rest = phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float wA = __fmul_rn(float(D2Q9::w(i)), rA[i]);
            const unsigned short q = E::enc(__fsub_rn(gv[i], wA));
            rest -= rebuild(q, wA);
            h[(8 + sl[i]) * NS + kk[i]] = q;
        }
        g0[kk[0]] = rest;  // slot 0 never moves and never bounces
        h[17 * NS + kk[0]] = ref_word(ownP);
        h[18 * NS + kk[0]] = ref_word(ownA);
    }
};

template <class ST>
struct IsDev {
    static constexpr bool value = false;
};
template <class H>
struct IsDev<Store16D<H>> {
    static constexpr bool value = true;
};

// ------------------------------------------------------------ helpers

__device__ __forceinline__ int wrap_x(int x, int nx) {
    // x within (-nx, 2nx) for all callers with nx >= 5 and halos <= 3 beyond
    // a 32-wide tile; fall back to a true modulo otherwise.
    if (x >= 0 && x < nx) return x;
    int r = x % nx;
    return r < 0 ? r + nx : r;
}

// Source row of a stencil position at global row y: periodic wrap, or the
// even mirror across walls at y = -1/2 and y = ny - 1/2, clamped into the
// domain (positions that far out are never read by an active cell).
__device__ __forceinline__ int src_row(int y, int ny, int wall) {
    if (!wall) {
        if (y >= 0 && y < ny) return y;
        int r = y % ny;
        return r < 0 ? r + ny : r;
    }
    int m = y < 0 ? -y - 1 : (y >= ny ? 2 * ny - 1 - y : y);
    return m < 0 ? 0 : (m >= ny ? ny - 1 : m);
}

// 9-point isotropic stencils on a shared-memory array with row stride W,
// centred at index c (reading of the "isotropic central scheme", Sec. 3):
//   grad = (1/cs2) sum w_i c_i chi(x + c_i)
//   lap  = (2/cs2) sum w_i [chi(x + c_i) - chi(x)]
template <class T>
__device__ __forceinline__ T lap9(const T *a, int c, int W) {
    const T C = a[c];
    const T ax = (a[c + 1] - C) + (a[c - 1] - C) + (a[c + W] - C) + (a[c - W] - C);
    const T dg = (a[c + W + 1] - C) + (a[c + W - 1] - C) + (a[c - W - 1] - C) + (a[c - W + 1] - C);
    return T(6) * (ax * T(1.0 / 9.0) + dg * T(1.0 / 36.0));
}

template <class T>
__device__ __forceinline__ void grad9(const T *a, int c, int W, T &gx, T &gy) {
    const T ne = a[c + W + 1], nw = a[c + W - 1], sw = a[c - W - 1], se = a[c - W + 1];
    gx = T(3) * ((a[c + 1] - a[c - 1]) * T(1.0 / 9.0) + ((ne - nw) + (se - sw)) * T(1.0 / 36.0));
    gy = T(3) * ((a[c + W] - a[c - W]) * T(1.0 / 9.0) + ((ne + nw) - (sw + se)) * T(1.0 / 36.0));
}

// Moments of one cell's populations: phi (Eq. 30), sum f, sum c f.
template <class T>
__device__ __forceinline__ void moments(const T f[9], const T g[9], T &phi, T &ps, T &jx, T &jy) {
    phi = g[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) phi += g[i];
    ps = f[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) ps += f[i];
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
}

// Shared-memory tile geometry for a 32 x TY tile.
template <class T, int TY>
struct Tile {
    static constexpr int TX = 32;
    static constexpr int PW = TX + 6, PH = TY + 6;  // phi, 3-cell halo
    static constexpr int MW = TX + 4, MH = TY + 4;  // mu, 2-cell halo
    static constexpr int QW = TX + 2, QH = TY + 2;  // sum f, j, p: 1-cell halo
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)PW * PH + (size_t)MW * MH + 4 * (size_t)QW * QH);
    T *phi, *mu, *ps, *jx, *jy, *p;
    __device__ __forceinline__ Tile(char *base) {
        phi = reinterpret_cast<T *>(base);
        mu = phi + PW * PH;
        ps = mu + MW * MH;
        jx = ps + QW * QH;
        jy = jx + QW * QH;
        p = jy + QW * QH;
    }
    __device__ __forceinline__ static int ip(int ly, int lx) { return (ly + 3) * PW + lx + 3; }
    __device__ __forceinline__ static int im(int ly, int lx) { return (ly + 2) * MW + lx + 2; }
    __device__ __forceinline__ static int iq(int ly, int lx) { return (ly + 1) * QW + lx + 1; }
};

// Local macroscopic state at a tile position within the 1-cell ring.
template <class T>
struct Macro {
    T phi, rho, mu, gphx, gphy, gmux, gmuy, lmu, Fx, Fy, ux, uy, p;
};

// F (Sec. 2: F_s = -phi grad mu, plus F_b), u (Eq. 31), p (Eq. 32).
template <class T, int TY>
__device__ __forceinline__ Macro<T> macro_at(const Tile<T, TY> &s, const KP<T> &P, int ly,
                                             int lx) {
    using TL = Tile<T, TY>;
    Macro<T> m;
    const int cp = TL::ip(ly, lx), cm = TL::im(ly, lx), cq = TL::iq(ly, lx);
    m.phi = s.phi[cp];
    m.rho = P.rhoB + (m.phi - P.phiB) * P.drho;
    m.mu = s.mu[cm];
    grad9(s.phi, cp, TL::PW, m.gphx, m.gphy);
    grad9(s.mu, cm, TL::MW, m.gmux, m.gmuy);
    m.lmu = lap9(s.mu, cm, TL::MW);
    m.Fx = -m.phi * m.gmux;
    m.Fy = -m.phi * m.gmuy - (m.rho - P.rhoref) * P.grav;
    const T irc = T(3) / m.rho;  // 1/(cs2 rho)
    m.ux = (s.jx[cq] + T(0.5 / 3.0) * m.Fx) * irc;
    m.uy = (s.jy[cq] + T(0.5 / 3.0) * m.Fy) * irc;
    const T udr = (m.ux * m.gphx + m.uy * m.gphy) * P.drho;
    m.p = s.ps[cq] + T(0.5 / 3.0) * (udr - P.gl * m.rho * m.lmu);
    return m;
}

// -------------------------------------------------------------- kernels


template <class T, class ST, int RPT, int MODE>
// MODE_ADJC in FP32 is held to 3 CTAs per SM (80 registers, 24 B spilled):
// at the compiler's 174 registers (1 CTA per SM) the adjoint's backward
// pass at 512^2 took 0.46 s, at 128 (2 CTAs) 0.376 s, at 80 0.370-0.374 s.
__global__ void __launch_bounds__(256, (MODE == MODE_ADJC && sizeof(T) == 4) ? 3 : 1)
k_step(const char *__restrict__ src, char *__restrict__ dst, const KP<T> P, FieldOut<T> out) {
    constexpr int TY = 8 * RPT;
    using TL = Tile<T, TY>;
    extern __shared__ __align__(16) char smem_raw[];
    TL s(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * TL::TX, y0 = blockIdx.y * TY;
    const int nx = P.nx, ny = P.ny, wall = P.wall;
    const long long NS = P.NS;

    // Phase 1a: owned cells, populations into registers, moments to smem.
    T fr[RPT][9], gr[RPT][9];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int ly = ty + 8 * r, lx = tx;
        const long long k = (long long)src_row(y0 + ly, ny, wall) * nx + wrap_x(x0 + lx, nx);
        if (!LBM_IDX_OK(P, k >= 0 && k < (long long)nx * ny, 5)) continue;
        ST::load(src, NS, k, fr[r], gr[r]);
        T phi, ps, jx, jy;
        moments(fr[r], gr[r], phi, ps, jx, jy);
        s.phi[TL::ip(ly, lx)] = phi;
        const int q = TL::iq(ly, lx);
        s.ps[q] = ps;
        s.jx[q] = jx;
        s.jy[q] = jy;
    }
    // Phase 1b: halo cells; phi on the 3-ring, sum f and j on the 1-ring.
    for (int j = tid; j < TL::PH * TL::PW; j += 256) {
        const int ry = j / TL::PW, rx = j - ry * TL::PW;
        const int ly = ry - 3, lx = rx - 3;
        if (ly >= 0 && ly < TY && lx >= 0 && lx < TL::TX) continue;
        const bool ring1 = (ly >= -1 && ly <= TY && lx >= -1 && lx <= TL::TX);
        const long long k = (long long)src_row(y0 + ly, ny, wall) * nx + wrap_x(x0 + lx, nx);
        if (!LBM_IDX_OK(P, k >= 0 && k < (long long)nx * ny, 5)) continue;
        if (ring1) {
            T f[9], g[9], phi, ps, jx, jy;
            ST::load(src, NS, k, f, g);
            moments(f, g, phi, ps, jx, jy);
            s.phi[j] = phi;
            const int q = TL::iq(ly, lx);
            s.ps[q] = ps;
            s.jx[q] = jx;
            s.jy[q] = jy;
        } else {
            s.phi[j] = ST::load_phi(src, NS, k);
        }
    }
    __syncthreads();

    // Phase 2: chemical potential (Eq. 5) on the 2-ring.  At a wall, a ghost
    // row takes mu of its mirror row (zero normal derivative).
    for (int j = tid; j < TL::MH * TL::MW; j += 256) {
        const int my = j / TL::MW, mx = j - my * TL::MW;
        int ly = my - 2;
        const int lx = mx - 2;
        if (wall) {
            const int gy = y0 + ly;
            if (gy < 0 || gy >= ny) {
                ly = src_row(gy, ny, 1) - y0;
                ly = ly < -2 ? -2 : (ly > TY + 1 ? TY + 1 : ly);
            }
        }
        const int c = TL::ip(ly, lx);
        const T ph = s.phi[c];
        s.mu[j] = P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) -
                  P.kappa * lap9(s.phi, c, TL::PW);
    }
    __syncthreads();

    // Phase 3: pressure (Eq. 32) on the 1-ring.  At a wall, a ghost row is
    // extrapolated linearly from the two rows inside.
    for (int j = tid; j < TL::QH * TL::QW; j += 256) {
        const int qy = j / TL::QW, qx = j - qy * TL::QW;
        const int ly = qy - 1, lx = qx - 1;
        const int gy = y0 + ly;
        T pv;
        if (!wall || (gy >= 0 && gy < ny)) {
            pv = macro_at<T, TY>(s, P, ly, lx).p;
        } else if (gy == -1) {
            pv = T(2) * macro_at<T, TY>(s, P, -y0, lx).p - macro_at<T, TY>(s, P, 1 - y0, lx).p;
        } else if (gy == ny) {
            pv = T(2) * macro_at<T, TY>(s, P, ny - 1 - y0, lx).p -
                 macro_at<T, TY>(s, P, ny - 2 - y0, lx).p;
        } else {
            pv = T(0);  // beyond a wall ghost row: never read by an active cell
        }
        s.p[j] = pv;
    }
    __syncthreads();

    // Phase 4: owned active cells.
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int ly = ty + 8 * r, lx = tx;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const Macro<T> m = macro_at<T, TY>(s, P, ly, lx);
        T gpx, gpy;
        grad9(s.p, TL::iq(ly, lx), TL::QW, gpx, gpy);
        const long long k = (long long)gy * nx + gx;
        const T pc = s.p[TL::iq(ly, lx)];
        if constexpr (MODE == MODE_ADJC) {
            const T q = (m.phi - P.phiA) * (m.phi - P.phiB) * (m.phi - P.phibar);
            const T lph = lap9(s.phi, TL::ip(ly, lx), TL::PW);
            AdjCell<T>::run(P, out, gx, gy, k, m, out.beta1x4 * q - out.kappa1 * lph, pc, gpx, gpy);
            continue;
        }
        if (MODE == MODE_FIELDS) {
            if (out.phi) out.phi[k] = m.phi;
            if (out.rho) out.rho[k] = m.rho;
            if (out.p) out.p[k] = pc;
            if (out.ux) out.ux[k] = m.ux;
            if (out.uy) out.uy[k] = m.uy;
            if (out.mu) out.mu[k] = m.mu;
            if (out.P) {
                // total pressure of Sec. 4.2: p0 - kappa phi lap phi + kappa |grad phi|^2/2 + p
                const T a = m.phi - P.phiA, b = m.phi - P.phiB;
                const T psi = P.beta * a * a * b * b;
                const T dpsi = P.beta4 * a * b * (m.phi - P.phibar);
                const T lph = lap9(s.phi, TL::ip(ly, lx), TL::PW);
                out.P[k] = m.phi * dpsi - psi - P.kappa * m.phi * lph +
                           T(0.5) * P.kappa * (m.gphx * m.gphx + m.gphy * m.gphy) + pc;
            }
            continue;
        }
        // Collision (Eqs. 22-29) with Gamma_i = 1 + s_i.
        const T ux = m.ux, uy = m.uy, rho = m.rho, phi = m.phi;
        const T grx = P.drho * m.gphx, gry = P.drho * m.gphy;
        const T uu = ux * ux + uy * uy;
        const T amu = P.alpha * m.mu;
        const T srcF = T(1.0 / 3.0) * rho * P.gl * m.lmu;       // cs2 rho gamma lambda lap mu
        const T gq = -T(3) * phi / rho;                           // -phi / (cs2 rho)
        const T dx = gpx - m.Fx, dy = gpy - m.Fy;
        T fv[9], gv[9];
        int sl[9];
        long long kk[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
            const T w = T(D2Q9::w(i));
            const T cu = T(cx) * ux + T(cy) * uy;
            const T si = T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
            const T wG = w * (T(1) + si);
            const T feq = w * (m.p + T(1.0 / 3.0) * rho * si);
            const T H = (i == 0) ? phi - T(1.0 - D2Q9::w(0)) * amu : w * amu;
            const T geq = H + w * phi * si;
            const T ex = T(cx) - ux, ey = T(cy) - uy;
            const T ws = w * si * T(1.0 / 3.0);
            const T Fi = ex * (wG * m.Fx + ws * grx) + ey * (wG * m.Fy + ws * gry) - w * srcF;
            const T Gi = gq * (ex * dx + ey * dy) * wG;
            const T f = fr[r][i], g = gr[r][i];
            T fs = f - (f - feq) * P.itf + P.pf * Fi;
            T gs = g - (g - geq) * P.itg + P.pg * Gi;
            // Streaming (left-hand sides of Eqs. 22-23), halfway bounce-back.
            const int yd = gy + cy;
            if (wall && (yd < 0 || yd >= ny)) {
                const T uw = yd < 0 ? P.uwb : P.uwt;
                const T cuw = T(cx) * uw;
                fs -= T(2) * w * rho * cuw;
                gs -= T(6) * w * phi * cuw;
                sl[i] = D2Q9::opp(i);
                kk[i] = k;
            } else {
                int xd = gx + cx;
                xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                int yy = yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd);
                sl[i] = i;
                kk[i] = (long long)yy * nx + xd;
            }
            fv[i] = fs;
            gv[i] = gs;
        }
        bool in = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) in = in && kk[i] >= 0 && kk[i] < (long long)nx * ny;
        if constexpr (!IsDev<ST>::value)
            if (LBM_IDX_OK(P, in, 2)) ST::store(dst, NS, sl, kk, fv, gv, phi);
    }
}

// Equilibrium initial state: p = 0, u = u0, mu from phi0 (Eq. 5),
// f = f^eq (Eq. 24), g = g^eq (Eqs. 25-27), written to level `lvl`.
template <class T, class ST>
__global__ void __launch_bounds__(256)
k_init(const T *__restrict__ phi0, const T *__restrict__ ux0, const T *__restrict__ uy0,
       char *__restrict__ lvl, const KP<T> P) {
    const int nx = P.nx, ny = P.ny;
    const long long N = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        T nb[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xx = wrap_x(x + D2Q9::cx(i), nx);
            const int yy = src_row(y + D2Q9::cy(i), ny, P.wall);
            nb[i] = phi0[(long long)yy * nx + xx];
        }
        const T ph = nb[0];
        T lap = T(0);
        {
            const T ax = (nb[1] - ph) + (nb[3] - ph) + (nb[2] - ph) + (nb[4] - ph);
            const T dg = (nb[5] - ph) + (nb[6] - ph) + (nb[7] - ph) + (nb[8] - ph);
            lap = T(6) * (ax * T(1.0 / 9.0) + dg * T(1.0 / 36.0));
        }
        const T mu = P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) - P.kappa * lap;
        const T rho = P.rhoB + (ph - P.phiB) * P.drho;
        const T ux = ux0 ? ux0[k] : T(0), uy = uy0 ? uy0[k] : T(0);
        const T uu = ux * ux + uy * uy;
        const T amu = P.alpha * mu;
        T fv[9], gv[9];
        int sl[9];
        long long kk[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const T w = T(D2Q9::w(i));
            const T cu = T(D2Q9::cx(i)) * ux + T(D2Q9::cy(i)) * uy;
            const T si = T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
            fv[i] = w * (T(1.0 / 3.0) * rho * si);
            const T H = (i == 0) ? ph - T(1.0 - D2Q9::w(0)) * amu : w * amu;
            gv[i] = H + w * ph * si;
            sl[i] = i;
            kk[i] = k;
        }
        if constexpr (IsDev<ST>::value) {
            // every population sits on its own cell: its references are
            // the cell's own p (0) and alpha mu, cut
            float rP[9], rA[9];
            const float A = ST::ref_cut(float(amu));
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                rP[i] = 0.0f;
                rA[i] = A;
            }
            ST::store(lvl, P.NS, sl, kk, fv, gv, ph, rP, rA, 0.0f, float(amu));
        } else {
            ST::store(lvl, P.NS, sl, kk, fv, gv, ph);
        }
    }
}

// Per-block partial sums (FP64) of rho and phi over the current level;
// fixed grid-stride order and a fixed shuffle tree make the result
// bitwise reproducible for a given grid size.
template <class T, class ST>
__global__ void __launch_bounds__(256)
k_mass_partial(const char *__restrict__ lvl, const KP<T> P, double *__restrict__ part) {
    const long long N = (long long)P.nx * P.ny;
    double sm = 0.0, sp = 0.0;
    const double rhoB = (double)P.rhoB, phiB = (double)P.phiB, drho = (double)P.drho;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const double ph = (double)ST::load_phi(lvl, P.NS, k);
        sp += ph;
        sm += rhoB + (ph - phiB) * drho;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sm += __shfl_down_sync(0xffffffffu, sm, o);
        sp += __shfl_down_sync(0xffffffffu, sp, o);
    }
    __shared__ double wm[8], wp[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        wm[wid] = sm;
        wp[wid] = sp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 8; ++i) {
            a += wm[i];
            b += wp[i];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// Laplace-diagnostic partial sums: inside sum/count, outside sum/count, A.
template <class T>
__global__ void __launch_bounds__(256)
k_laplace_partial(const T *__restrict__ Ptot, const T *__restrict__ phi, const KP<T> P, double xc,
                  double yc, double rin, double rout, double *__restrict__ part) {
    const int nx = P.nx, ny = P.ny;
    const long long N = (long long)nx * ny;
    double v[5] = {0, 0, 0, 0, 0};
    const double phiB = (double)P.phiB, dphi = (double)(P.phiA - P.phiB);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        double dx = fabs(x - xc), dy = fabs(y - yc);
        if (dx > 0.5 * nx) dx = nx - dx;
        if (dy > 0.5 * ny) dy = ny - dy;
        const double r = sqrt(dx * dx + dy * dy);
        const double pv = (double)Ptot[k];
        if (r < rin) { v[0] += pv; v[1] += 1.0; }
        if (r > rout) { v[2] += pv; v[3] += 1.0; }
        v[4] += ((double)phi[k] - phiB) / dphi;
    }
    __shared__ double red[5][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double a = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[q][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double a = 0.0;
        for (int i = 0; i < 8; ++i) a += red[threadIdx.x][i];
        part[5 * blockIdx.x + threadIdx.x] = a;
    }
}

// Second stage of the reductions: the `width` (<= 8) totals of `nblocks`
// per-block partial records, in a fixed order, by one block of 256
// threads.  Thread t sums records t, t + 256, ... in ascending order, each
// warp folds its 32 sums by shuffles, and thread j adds the 8 warp sums of
// total j in warp order.  ADD: out[j] += total, else out[j] = total.
template <bool ADD>
__device__ __forceinline__ void fold_partials(const double *__restrict__ part, int nblocks, int width,
                                              double *__restrict__ out) {
    __shared__ double ws[8][8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int j = 0; j < width; ++j) {
        double a = 0.0;
        for (int b = t; b < nblocks; b += 256) a += part[width * b + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) ws[wid][j] = a;
    }
    __syncthreads();
    if (t < width) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w][t];
        if (ADD) out[t] += s;
        else out[t] = s;
    }
}

static __global__ void __launch_bounds__(256) k_reduce_final(const double *__restrict__ part, int nblocks,
                                                             int width, double *__restrict__ out) {
    fold_partials<false>(part, nblocks, width, out);
}

}  // namespace lbm
