// lbm_strip.cuh — the streaming form of the time step, for grids whose nx
// is a multiple of 8 (and whose level fits 32-bit element offsets).
//
// Same arithmetic as k_step (lbm_kernels.cuh), reorganised so that the
// radius-3 coupling of the step (grad p <- p <- lap mu <- lap phi) costs
// an x-halo only:
//   * A CTA of SW threads owns a column strip x0 .. x0+SW-1 and a segment
//     of rows ys .. ye-1, and marches up through y.  Iteration y
//       1. phi at row y+3 from the g populations of that row,
//       3. mu  at row y+2 (Eq. 5),
//       4. p   at row y+1 (Eq. 32) from sum f and j of that row's f
//          populations; each thread keeps u (Eq. 31), F, lap mu and
//          grad phi of its own column in registers for the next iteration,
//       5. collides row y (Eqs. 22-29) and pushes it to the other level.
//     Rows of phi, mu and p live in small shared-memory rings (4, 3, 3
//     rows: the rows live at iteration y).
//   * Population rows are copied global -> shared with cp.async (16-byte
//     chunks, L2 only) DEPTH rows ahead of use, so DRAM traffic overlaps the
//     arithmetic of the rows in flight.  Every population is read from DRAM
//     once (plus the 2 x HP halo columns and 6 warm-up rows per segment,
//     which mostly hit L2) and written once.
//   * Walls: ghost rows of phi come from loading the mirror row; a ghost mu
//     row copies its mirror row when that row exists; the ghost p row is
//     extrapolated from the two rows inside (same rules as k_step).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; maps are encoded on the host)

#include <type_traits>

#include "lbm_internal.h"
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

// Tensor-tile staging (FP32 single domains, strips that do not wrap in x):
// one thread copies a whole population row (9 slots x 1 row x LW columns,
// one box of the level's 3-D tensor map) into shared memory with a TMA
// load that completes on the ring slot's mbarrier; every thread waits on
// that barrier's phase before reading the row.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// one arrival that also announces `bytes` of transfer still to land
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity` to complete: false when it
// has not after about one second (the device's global nanosecond timer),
// or after kMbarTries polls at most, so that no kernel waits forever on a
// copy that never lands.
constexpr int kMbarTries = 1 << 24;
constexpr unsigned long long kMbarWaitNs = 1000000000ULL;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kMbarTries; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > kMbarWaitNs) return false;
    }
    return false;
}
// 3-D tile load: box at (x, y, z) of the map into shared memory at dst.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, unsigned bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
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

__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }

// Threads of a strip CTA of SW columns: SW itself when SW is a multiple of
// the warp size (each step's halo columns then take an extra pass of one
// warp), otherwise enough whole warps to cover SW + 6 columns, so that every
// step (at most 3 halo columns per side) is a single pass.
__host__ __device__ constexpr int strip_threads(int SW) {
    return SW % 32 == 0 ? SW : (SW + 6 + 31) / 32 * 32;
}

// Shared-memory row buffers of the populations, per storage type.  A row
// buffer holds columns x0-HP .. x0+SW+HP-1 of every slot; the async copy of
// a row is described once per thread (which 16-byte chunks it copies) and
// replayed for every row with only the row offset changing.
template <class ST, int SW>
struct StripRow;

template <class T, int SW>
struct StripRow<PlainStore<T>, SW> {
    using C = T;
    static constexpr int HP = 4;               // halo columns loaded each side
    static constexpr int LW = SW + 2 * HP;     // row width
    static constexpr int CE = 16 / sizeof(T);  // elements per 16-byte chunk
    static constexpr int CPS = LW / CE;        // chunks per slot
    static constexpr int TOTAL = 9 * CPS;      // chunks of one f row (or g row)
    static constexpr int NT = strip_threads(SW);
    static constexpr int NCH = (TOTAL + NT - 1) / NT;
    static constexpr size_t fbytes = (size_t)9 * LW * sizeof(T);  // f_0..f_8
    static constexpr size_t gbytes = (size_t)9 * LW * sizeof(T);  // g_0..g_8
    static bool idx32_ok(long long NS) { return 18 * NS < (1LL << 31); }

    // A thread copies the same chunks of every f row and of every g row.
    struct Desc {
        int goff[NCH], soff[NCH];
        int gslot;  // element offset of the g slots: 9 NS
    };
    // Only the chunks covering the strip's active columns and their halo
    // (x_start .. x_start + need - 1) are copied: a domain narrower than the
    // strip would otherwise load the same row several times over.
    __device__ __forceinline__ static void describe(Desc &d, int t, long long NS, int x_start,
                                                    int nx, int need) {
        d.gslot = 9 * (int)NS;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const int j = t + k * NT;
            const int c0 = (j % CPS) * CE;
            if (j < TOTAL && c0 < need) {
                const int sl = j / CPS, c = j - sl * CPS;
                d.goff[k] = sl * (int)NS + wrap_any(x_start + c * CE, nx);
                d.soff[k] = sl * LW + c * CE;
            } else {
                d.goff[k] = -1;
                d.soff[k] = 0;
            }
        }
    }
    __device__ __forceinline__ static void issue_f(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const T *g = reinterpret_cast<const T *>(lvl);
        T *s = reinterpret_cast<T *>(sbuf);
#pragma unroll
        for (int k = 0; k < NCH; ++k)
            if (d.goff[k] >= 0) cp_async16(s + d.soff[k], g + (d.goff[k] + rowbase));
    }
    __device__ __forceinline__ static void issue_g(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const T *g = reinterpret_cast<const T *>(lvl) + d.gslot;
        T *s = reinterpret_cast<T *>(sbuf);
#pragma unroll
        for (int k = 0; k < NCH; ++k)
            if (d.goff[k] >= 0) cp_async16(s + d.soff[k], g + (d.goff[k] + rowbase));
    }
    __device__ __forceinline__ static void read_f(const char *fbuf, int c, C f[9]) {
        const T *s = reinterpret_cast<const T *>(fbuf);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = s[i * LW + c];
    }
    __device__ __forceinline__ static void read_g(const char *gbuf, int c, C g[9]) {
        const T *s = reinterpret_cast<const T *>(gbuf);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = s[i * LW + c];
    }
    // Tensor-tile rows (one map per level: x, row, 18 slots): the g row is
    // the box at slot 9, the f row the box at slot 0.
    static constexpr int NMAP = 1;
    static constexpr unsigned TMA_GB = (unsigned)(9 * LW * sizeof(T)), TMA_FB = TMA_GB;
    __device__ __forceinline__ static void tma_g(unsigned dst, const CUtensorMap *m, unsigned bar,
                                                 int x, int row) {
        tma_load_3d(dst, m, bar, x, row, 9);
    }
    __device__ __forceinline__ static void tma_f(unsigned dst, const CUtensorMap *m, unsigned bar,
                                                 int x, int row) {
        tma_load_3d(dst, m, bar, x, row, 0);
    }
    // Interior push: slot i of cell kb + cy_i nx + cx_i, 32-bit offsets.
    __device__ __forceinline__ static void store_fast(char *lvl, int NS, int nx, int kb,
                                                      const C fv[9], const C gv[9], C phi) {
        T *b = reinterpret_cast<T *>(lvl) + kb;
#pragma unroll
        for (int i = 0; i < 9; ++i) b[i * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = fv[i];
        b[9 * NS] = PlainStore<T>::g0_value(gv, phi);
#pragma unroll
        for (int i = 1; i < 9; ++i) b[(9 + i) * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = gv[i];
    }
};

template <class H, int SW>
struct StripRow<Store16<H>, SW> {
    using C = float;
    using E = HalfStore<H>;
    static constexpr int HP = 8;  // 8 halves per 16-byte chunk
    static constexpr int LW = SW + 2 * HP;
    static constexpr int CH = LW / 8, C0 = LW / 4;  // chunks per half slot, of the g_0 row
    static constexpr int TF = 9 * CH;               // f row: half slots 0..8
    static constexpr int TG = C0 + 8 * CH;          // g row: g_0 floats, half slots 9..16
    static constexpr int NT = strip_threads(SW);
    static constexpr int NF = (TF + NT - 1) / NT, NG = (TG + NT - 1) / NT;
    // a g row holds the g_0 floats, padded to a 128-byte multiple so that
    // its half slots start on a tensor-tile boundary, then half slots 9..16
    static constexpr int G0B = (LW * 4 + 127) / 128 * 128;
    static constexpr size_t fbytes = (size_t)9 * LW * 2;
    static constexpr size_t gbytes = (size_t)G0B + (size_t)8 * LW * 2;
    // offsets count halves from the level base: half slot s starts at half
    // index (2 + s) NS, after the NS floats of g_0
    static bool idx32_ok(long long NS) { return 19 * NS < (1LL << 31); }
    // Tensor-tile rows, three maps per level: [0] the 17 half slots with
    // boxes of 9 slots (the f row: slots 0..8), [1] the same with boxes of 8
    // (the g row's slots 9..16), [2] the g_0 floats (one slot).
    static constexpr int NMAP = 3;
    static constexpr unsigned TMA_GB = (unsigned)(LW * 4 + 8 * LW * 2), TMA_FB = (unsigned)(9 * LW * 2);
    __device__ __forceinline__ static void tma_g(unsigned dst, const CUtensorMap *m, unsigned bar,
                                                 int x, int row) {
        tma_load_3d(dst, m + 2, bar, x, row, 0);
        tma_load_3d(dst + G0B, m + 1, bar, x, row, 9);
    }
    __device__ __forceinline__ static void tma_f(unsigned dst, const CUtensorMap *m, unsigned bar,
                                                 int x, int row) {
        tma_load_3d(dst, m, bar, x, row, 0);
    }

    struct Desc {
        int foff[NF], fso[NF];      // f chunks: global half offset, smem half offset
        int goff[NG], gso[NG];      // g chunks: global offset (floats for g_0, else halves)
        unsigned gflt;              // bit k: chunk k of the g row is a g_0 (float) chunk
    };
    __device__ __forceinline__ static void describe(Desc &d, int t, long long NS, int x_start,
                                                    int nx, int need) {
        const int ns = (int)NS;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int j = t + k * NT;
            if (j < TF && (j % CH) * 8 < need) {
                const int sl = j / CH, c = j - sl * CH;
                d.foff[k] = (2 + sl) * ns + wrap_any(x_start + c * 8, nx);
                d.fso[k] = sl * LW + c * 8;
            } else {
                d.foff[k] = -1;
                d.fso[k] = 0;
            }
        }
        d.gflt = 0;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const int j = t + k * NT;
            if (j < C0 && j * 4 < need) {
                d.goff[k] = wrap_any(x_start + j * 4, nx);
                d.gso[k] = j * 16;  // bytes
                d.gflt |= 1u << k;
            } else if (j >= C0 && j < TG && ((j - C0) % CH) * 8 < need) {
                const int jj = j - C0;
                const int sl = jj / CH, c = jj - sl * CH;
                d.goff[k] = (2 + 9 + sl) * ns + wrap_any(x_start + c * 8, nx);
                d.gso[k] = G0B + (sl * LW + c * 8) * 2;  // bytes
            } else {
                d.goff[k] = -1;
                d.gso[k] = 0;
            }
        }
    }
    __device__ __forceinline__ static void issue_f(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl);
        unsigned short *sh = reinterpret_cast<unsigned short *>(sbuf);
#pragma unroll
        for (int k = 0; k < NF; ++k)
            if (d.foff[k] >= 0) cp_async16(sh + d.fso[k], h + (d.foff[k] + rowbase));
    }
    __device__ __forceinline__ static void issue_g(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl);
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            if (d.goff[k] < 0) continue;
            const void *src = ((d.gflt >> k) & 1u) ? static_cast<const void *>(g0 + (d.goff[k] + rowbase))
                                                   : static_cast<const void *>(h + (d.goff[k] + rowbase));
            cp_async16(sbuf + d.gso[k], src);
        }
    }
    __device__ __forceinline__ static void read_f(const char *fbuf, int c, C f[9]) {
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(fbuf);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = E::dec(sh[i * LW + c]);
    }
    __device__ __forceinline__ static void read_g(const char *gbuf, int c, C g[9]) {
        const float *s0 = reinterpret_cast<const float *>(gbuf);
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(gbuf + G0B);
        g[0] = s0[c];
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = E::dec(sh[(i - 1) * LW + c]);
    }
    __device__ __forceinline__ static void store_fast(char *lvl, int NS, int nx, int kb,
                                                      const C fv[9], const C gv[9], C phi) {
        float *g0 = reinterpret_cast<float *>(lvl);
        unsigned short *h = reinterpret_cast<unsigned short *>(lvl + (size_t)NS * 4) + kb;
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = E::enc(fv[i]);
        float rest = phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const unsigned short q = E::enc(gv[i]);
            rest -= E::dec(q);
            h[(8 + i) * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = q;
        }
        g0[kb] = rest;
    }
};

// Deviation storage: an f row carries f_0..f_8 and the reference word P
// (10 half slots), a g row g_0 (floats), g_1..g_8 and the reference word A
// (9 half slots).  Reads rebuild the populations from the references of
// the row's own cells; pushes take the references of the destination
// cells (rP, rA, already cut) and write this cell's own words.
template <class H, int SW>
struct StripRow<Store16D<H>, SW> {
    using C = float;
    using ST = Store16D<H>;
    using E = HalfStore<H>;
    static constexpr int HP = 8;
    static constexpr int LW = SW + 2 * HP;
    static constexpr int CH = LW / 8, C0 = LW / 4;
    static constexpr int TF = 10 * CH;         // f row: f_0..f_8, P
    static constexpr int TG = C0 + 9 * CH;     // g row: g_0 floats, g_1..g_8, A
    static constexpr int NT = strip_threads(SW);
    static constexpr int NF = (TF + NT - 1) / NT, NG = (TG + NT - 1) / NT;
    static constexpr size_t fbytes = (size_t)10 * LW * 2;
    static constexpr size_t gbytes = (size_t)LW * 4 + (size_t)9 * LW * 2;
    static bool idx32_ok(long long NS) { return 21 * NS < (1LL << 31); }

    struct Desc {
        int foff[NF], fso[NF];
        int goff[NG], gso[NG];
        unsigned gflt;
    };
    // global half slot of f row slot sl (0..9) and of g row half slot sl (0..8)
    __device__ __forceinline__ static int fslot(int sl) { return sl < 9 ? sl : 17; }
    __device__ __forceinline__ static int gslot(int sl) { return sl < 8 ? 9 + sl : 18; }
    __device__ __forceinline__ static void describe(Desc &d, int t, long long NS, int x_start,
                                                    int nx, int need) {
        const int ns = (int)NS;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            const int j = t + k * NT;
            if (j < TF && (j % CH) * 8 < need) {
                const int sl = j / CH, c = j - sl * CH;
                d.foff[k] = (2 + fslot(sl)) * ns + wrap_any(x_start + c * 8, nx);
                d.fso[k] = sl * LW + c * 8;
            } else {
                d.foff[k] = -1;
                d.fso[k] = 0;
            }
        }
        d.gflt = 0;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const int j = t + k * NT;
            if (j < C0 && j * 4 < need) {
                d.goff[k] = wrap_any(x_start + j * 4, nx);
                d.gso[k] = j * 16;
                d.gflt |= 1u << k;
            } else if (j >= C0 && j < TG && ((j - C0) % CH) * 8 < need) {
                const int jj = j - C0;
                const int sl = jj / CH, c = jj - sl * CH;
                d.goff[k] = (2 + gslot(sl)) * ns + wrap_any(x_start + c * 8, nx);
                d.gso[k] = LW * 4 + (sl * LW + c * 8) * 2;
            } else {
                d.goff[k] = -1;
                d.gso[k] = 0;
            }
        }
    }
    __device__ __forceinline__ static void issue_f(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl);
        unsigned short *sh = reinterpret_cast<unsigned short *>(sbuf);
#pragma unroll
        for (int k = 0; k < NF; ++k)
            if (d.foff[k] >= 0) cp_async16(sh + d.fso[k], h + (d.foff[k] + rowbase));
    }
    __device__ __forceinline__ static void issue_g(const Desc &d, char *sbuf, const char *lvl,
                                                   int rowbase) {
        const float *g0 = reinterpret_cast<const float *>(lvl);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(lvl);
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            if (d.goff[k] < 0) continue;
            const void *src = ((d.gflt >> k) & 1u) ? static_cast<const void *>(g0 + (d.goff[k] + rowbase))
                                                   : static_cast<const void *>(h + (d.goff[k] + rowbase));
            cp_async16(sbuf + d.gso[k], src);
        }
    }
    __device__ __forceinline__ static void read_f(const char *fbuf, int c, C f[9]) {
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(fbuf);
        const float Pr = ST::ref_value(sh[9 * LW + c]);
        const float w0 = __fmul_rn(float(D2Q9::w(0)), Pr), w1 = __fmul_rn(float(D2Q9::w(1)), Pr),
                    w5 = __fmul_rn(float(D2Q9::w(5)), Pr);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = ST::rebuild(sh[i * LW + c], i == 0 ? w0 : (i < 5 ? w1 : w5));
    }
    __device__ __forceinline__ static void read_g(const char *gbuf, int c, C g[9]) {
        const float *s0 = reinterpret_cast<const float *>(gbuf);
        const unsigned short *sh = reinterpret_cast<const unsigned short *>(gbuf + (size_t)LW * 4);
        const float Ar = ST::ref_value(sh[8 * LW + c]);
        const float w1 = __fmul_rn(float(D2Q9::w(1)), Ar), w5 = __fmul_rn(float(D2Q9::w(5)), Ar);
        g[0] = s0[c];
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = ST::rebuild(sh[(i - 1) * LW + c], i < 5 ? w1 : w5);
    }
    __device__ __forceinline__ static void store_fast(char *lvl, int NS, int nx, int kb,
                                                      const C fv[9], const C gv[9], C phi,
                                                      const float rP[9], const float rA[9],
                                                      float ownP, float ownA) {
        float *g0 = reinterpret_cast<float *>(lvl);
        unsigned short *h = reinterpret_cast<unsigned short *>(lvl + (size_t)NS * 4) + kb;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float wP = __fmul_rn(float(D2Q9::w(i)), rP[i]);
            h[i * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = E::enc(__fsub_rn(fv[i], wP));
        }
        float rest = phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float wA = __fmul_rn(float(D2Q9::w(i)), rA[i]);
            const unsigned short q = E::enc(__fsub_rn(gv[i], wA));
            rest -= ST::rebuild(q, wA);
            h[(8 + i) * NS + D2Q9::cy(i) * nx + D2Q9::cx(i)] = q;
        }
        g0[kb] = rest;
        h[17 * NS] = ST::ref_word(ownP);
        h[18 * NS] = ST::ref_word(ownA);
    }
};

// Shared-memory layout of one strip CTA.
template <class T, class ST, int SW, int DEPTH>
struct StripSmem {
    using SR = StripRow<ST, SW>;
    using Tp = T;
    static constexpr int HP = SR::HP;
    static constexpr int LW = SR::LW;
    // g rows are read 3 iterations after they arrive (phi, then collision),
    // f rows 1 iteration after (sum f and j, then collision): separate rings.
    // FP32 plain storage on one-pass strips keeps each thread's own f values
    // in registers from the moments (step 4) to the next iteration's
    // collision, so its f ring holds only the row being summed and the rows
    // in flight (one row less: 6 CTAs per SM instead of 5); F1 is the ring
    // index of f row y+1.  At 128-column strips the carry frees no CTA slot
    // and only adds moves, so it is off there.
    static constexpr bool FCARRY =
        std::is_same<ST, PlainStore<float>>::value && strip_threads(SW) != SW;
    static constexpr int NBG = DEPTH + 4, NBF = FCARRY ? DEPTH + 1 : DEPTH + 2;
    static constexpr int F1 = FCARRY ? 0 : 1;
    // rows live at iteration y: phi y..y+3, mu y..y+2 (and y-1 with the
    // deviation storage, whose pushes need the destinations' mu), p
    // y-1..y+1; mu[MU0 + k] holds row y+k
    static constexpr bool DEV = IsDev<ST>::value;
    static constexpr int RPHI = 4, RMU = DEV ? 4 : 3, RP = 3, MU0 = RMU - 3;
    static constexpr int WPHI = SW + 6, WMU = SW + 4, WQ = SW + 2;
    // row buffers on 128-byte boundaries (tensor-tile destinations)
    static constexpr size_t gb = (SR::gbytes + 127) / 128 * 128;
    static constexpr size_t fb = (SR::fbytes + 127) / 128 * 128;
    static constexpr size_t pop_bytes = gb * NBG + fb * NBF;
    static constexpr size_t fld_elems =
        (size_t)RPHI * WPHI + (size_t)RMU * WMU + (size_t)RP * WQ;
    static constexpr size_t bytes = pop_bytes + fld_elems * sizeof(T);
    // Order in shared memory: NBG g rows, NBF f rows, then the phi, mu and
    // p rings (RingSlots holds the offsets).
    // With the f carry, and for the deviation storage, the CTAs per SM that
    // the shared memory allows (228 KB per SM, 1 KB per CTA reserved) become
    // the register budget the compiler is held to, so that registers do not
    // become the tighter limit; otherwise (0) the compiler's own choice
    // stands.  (The deviation kernels would take 96 registers, 5 CTAs per
    // SM; at 80 they spill 16-20 bytes and measured 1% (FP16) and 3% (BF16)
    // faster with 6.)
    static constexpr int MINB = (FCARRY || DEV) ? int(233472 / (bytes + 1024)) : 0;
    // tensor-tile staging: the rows issued in one iteration (a g row and an
    // f row) complete on one mbarrier; DEPTH + 1 barriers after the rings
    // are reused in turn.  The row buffers of a TMA load must start on
    // 128-byte boundaries.
    static constexpr int NBAR = DEPTH + 1;
    static constexpr size_t bar_off = (bytes + 7) / 8 * 8;
    static constexpr size_t bytes_tma = bar_off + 8 * (size_t)NBAR;
    static constexpr bool TMA_ROWS = gb % 128 == 0 && fb % 128 == 0;
};

// The ring slots of the rows live at iteration y, as byte offsets into the
// CTA's shared memory (column 0 of the strip for the field rings):
// g[k], f[k], ph[k], mu[k] hold row y+k and p[k] row y-1+k.  Advancing y
// rotates the slots (register moves) instead of reducing row indices
// modulo the ring sizes at every access.
template <class SM>
struct RingSlots {
    using T = typename SM::Tp;
    int g[SM::NBG], f[SM::NBF], ph[SM::RPHI], mu[SM::RMU], p[SM::RP];
    __device__ __forceinline__ RingSlots() {
        constexpr int E = sizeof(T);
        constexpr int b_mu = (int)SM::pop_bytes + SM::RPHI * SM::WPHI * E;
        constexpr int b_p = b_mu + SM::RMU * SM::WMU * E;
#pragma unroll
        for (int k = 0; k < SM::NBG; ++k) g[k] = k * (int)SM::gb;
#pragma unroll
        for (int k = 0; k < SM::NBF; ++k) f[k] = (int)(SM::gb * SM::NBG) + k * (int)SM::fb;
#pragma unroll
        for (int k = 0; k < SM::RPHI; ++k) ph[k] = (int)SM::pop_bytes + (k * SM::WPHI + 3) * E;
#pragma unroll
        for (int k = 0; k < SM::RMU; ++k) mu[k] = b_mu + (k * SM::WMU + 2) * E;
#pragma unroll
        for (int k = 0; k < SM::RP; ++k) p[k] = b_p + (k * SM::WQ + 1) * E;
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
        rot(ph);
        rot(mu);
        rot(p);
    }
};

// Row of the level buffer that holds global row y.  The whole domain wraps
// rows outside 0..ny-1 (periodic) or mirrors them (walls).  A slab holds
// rows y0 .. y0+rows-1, whose ghost rows its neighbours filled in (or, at a
// wall, mirrors into its own rows); rows beyond that feed only warm-up
// results that are never used, so they are clamped to the buffer.
template <bool SLAB, class T>
__device__ __forceinline__ int buf_row(const KP<T> &P, int y) {
    if (!SLAB) return src_row(y, P.ny, P.wall);
    int m = y;
    if (P.wall) m = y < 0 ? -y - 1 : (y >= P.ny ? 2 * P.ny - 1 - y : y);
    const int l = m - P.y0;
    return l < 0 ? 0 : (l >= P.rows ? P.rows - 1 : l);
}

// Column loop of one step: columns -h .. SW+h-1.  Every thread takes column
// t - h; the 2h columns past SW-h are taken by the first 2h lanes of warp
// `xw` (a different warp per step), so no warp carries every extra pass.
template <int SW, int H, int XW, class F>
__device__ __forceinline__ void columns(int t, F &&fn) {
    if constexpr (strip_threads(SW) >= SW + 2 * H) {
        if (t < SW + 2 * H) fn(t - H);  // one pass
    } else {
        fn(t - H);
        constexpr int NW = SW / 32;
        if ((t >> 5) == (XW % NW) && (t & 31) < 2 * H) fn(SW - H + (t & 31));
    }
}

// What the collision of one cell needs (Eqs. 22-29): phi, mu, p, rho,
// u (Eq. 31), F (Eq. 30 with the body force), lap mu, grad phi and grad p.
template <class T>
struct CellState {
    T phi, mu, p, rho, ux, uy, Fx, Fy, lm, gphx, gphy, gpx, gpy;
};

// BGK collision of one cell with Gamma_i = 1 + s_i: post-collision f*_i
// (Eqs. 22, 24, 28) and g*_i (Eqs. 23, 25, 27, 29), direction by direction.
// With Z = F + grad(rho)/3 and D = grad p - F,
//   F_i-term:  (c_i - u).F + s_i (c_i - u).Z
//   G_i-term:  (1 + s_i) (c_i - u).D
template <class T>
__device__ __forceinline__ void collide(const KP<T> &P, const CellState<T> &c, const T f[9],
                                        const T g[9], T fv[9], T gv[9]) {
    const T c3 = T(1.0 / 3.0);
    const T ux = c.ux, uy = c.uy, Fx = c.Fx, Fy = c.Fy;
    const T gr3x = (c3 * P.drho) * c.gphx;  // grad rho / 3
    const T gr3y = (c3 * P.drho) * c.gphy;
    const T Zx = Fx + gr3x, Zy = Fy + gr3y;
    const T dx = c.gpx - Fx, dy = c.gpy - Fy;
    const T uu15 = T(1.5) * (ux * ux + uy * uy);
    const T uF = ux * Fx + uy * Fy;
    const T uZ = ux * Zx + uy * Zy;
    const T uD = ux * dx + uy * dy;
    const T Q = P.pg * (T(-3) * c.phi * rcp_fast(c.rho));  // pg * (-phi / (cs2 rho))
    const T Bf = P.itf * (c3 * c.rho);                       // itf cs2 rho
    const T Kf = P.itf * c.p - P.pf * (c3 * c.rho * P.gl * c.lm);
    const T omf = T(1) - P.itf, omg = T(1) - P.itg;
    const T phg = P.itg * c.phi;
    const T Ag = P.itg * P.alpha * c.mu;                     // itg alpha mu
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
        const T w = T(D2Q9::w(i));
        const T cu = T(cx) * ux + T(cy) * uy;
        const T si = cu * (T(3) + T(4.5) * cu) - uu15;  // s_i (Eq. 26)
        const T eF = (T(cx) * Fx + T(cy) * Fy) - uF;    // (c_i - u).F
        const T eZ = (T(cx) * Zx + T(cy) * Zy) - uZ;    // (c_i - u).Z
        const T eD = (T(cx) * dx + T(cy) * dy) - uD;    // (c_i - u).D
        fv[i] = omf * f[i] + w * (Kf + Bf * si + P.pf * (eF + si * eZ));
        const T Hg = (i == 0) ? (phg - T(1.0 - D2Q9::w(0)) * Ag) * T(1.0 / D2Q9::w(0)) : Ag;
        gv[i] = omg * g[i] + w * (Hg + phg * si + Q * (eD + si * eD));
    }
}

// FP32: the same arithmetic with directions (1,2), (3,4), (5,6), (7,8) in
// the two lanes of packed f32x2 operations.  Direction 3 is -1 times
// direction 1 (4 of 2, 7 of 5, 8 of 6), so both pairs of a class share the
// products c_i.u, c_i.F, c_i.Z, c_i.D and differ in sign only.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

template <int SGN>
__device__ __forceinline__ void collide_pair(float2 cu, float2 cF, float2 cZ, float2 cD, float w,
                                             float2 mu15, float2 muF, float2 muZ, float2 muD,
                                             float2 Kf, float2 Bf, float2 pf, float2 omf,
                                             float2 Ag, float2 phg, float2 Q, float2 omg,
                                             float2 f, float2 g, float2 &fo, float2 &go) {
    const float2 sg = bc2(float(SGN));
    // s_i = (SGN cu)(3 + 4.5 SGN cu) - 1.5 u.u = cu (4.5 cu + 3 SGN) - 1.5 u.u
    const float2 si = __ffma2_rn(cu, __ffma2_rn(cu, bc2(4.5f), bc2(3.0f * SGN)), mu15);
    const float2 eF = __ffma2_rn(cF, sg, muF);
    const float2 eZ = __ffma2_rn(cZ, sg, muZ);
    const float2 eD = __ffma2_rn(cD, sg, muD);
    const float2 w2 = bc2(w);
    float2 a = __ffma2_rn(Bf, si, Kf);
    a = __ffma2_rn(pf, __ffma2_rn(si, eZ, eF), a);
    fo = __ffma2_rn(omf, f, __fmul2_rn(w2, a));
    float2 b = __ffma2_rn(phg, si, Ag);
    b = __ffma2_rn(Q, __ffma2_rn(si, eD, eD), b);
    go = __ffma2_rn(omg, g, __fmul2_rn(w2, b));
}

__device__ __forceinline__ void collide(const KP<float> &P, const CellState<float> &c,
                                        const float f[9], const float g[9], float fv[9],
                                        float gv[9]) {
    const float c3 = 1.0f / 3.0f;
    const float ux = c.ux, uy = c.uy, Fx = c.Fx, Fy = c.Fy;
    const float Zx = Fx + (c3 * P.drho) * c.gphx, Zy = Fy + (c3 * P.drho) * c.gphy;
    const float dx = c.gpx - Fx, dy = c.gpy - Fy;
    const float uu15 = 1.5f * (ux * ux + uy * uy);
    const float uF = ux * Fx + uy * Fy;
    const float uZ = ux * Zx + uy * Zy;
    const float uD = ux * dx + uy * dy;
    const float Q = P.pg * (-3.0f * c.phi * rcp_fast(c.rho));
    const float Bf = P.itf * (c3 * c.rho);
    const float Kf = P.itf * c.p - P.pf * (c3 * c.rho * P.gl * c.lm);
    const float omf = 1.0f - P.itf, omg = 1.0f - P.itg;
    const float phg = P.itg * c.phi;
    const float Ag = P.itg * P.alpha * c.mu;
    // direction 0 (c_0 = 0)
    {
        const float w = float(D2Q9::w(0));
        const float si = -uu15;
        fv[0] = omf * f[0] + w * (Kf + Bf * si + P.pf * (-uF - si * uZ));
        const float H0 = (phg - float(1.0 - D2Q9::w(0)) * Ag) * float(1.0 / D2Q9::w(0));
        gv[0] = omg * g[0] + w * (H0 + phg * si + Q * (-uD - si * uD));
    }
    const float2 mu15 = bc2(-uu15), muF = bc2(-uF), muZ = bc2(-uZ), muD = bc2(-uD);
    const float2 Kf2 = bc2(Kf), Bf2 = bc2(Bf), pf2 = bc2(P.pf), omf2 = bc2(omf);
    const float2 Ag2 = bc2(Ag), phg2 = bc2(phg), Q2 = bc2(Q), omg2 = bc2(omg);
    float2 fo, go;
    // axis directions: (1,2) = +(e_x, e_y), (3,4) = -(e_x, e_y)
    {
        const float2 cu = make_float2(ux, uy), cF = make_float2(Fx, Fy);
        const float2 cZ = make_float2(Zx, Zy), cD = make_float2(dx, dy);
        const float w = float(D2Q9::w(1));
        collide_pair<1>(cu, cF, cZ, cD, w, mu15, muF, muZ, muD, Kf2, Bf2, pf2, omf2, Ag2, phg2, Q2,
                        omg2, make_float2(f[1], f[2]), make_float2(g[1], g[2]), fo, go);
        fv[1] = fo.x, fv[2] = fo.y, gv[1] = go.x, gv[2] = go.y;
        collide_pair<-1>(cu, cF, cZ, cD, w, mu15, muF, muZ, muD, Kf2, Bf2, pf2, omf2, Ag2, phg2, Q2,
                         omg2, make_float2(f[3], f[4]), make_float2(g[3], g[4]), fo, go);
        fv[3] = fo.x, fv[4] = fo.y, gv[3] = go.x, gv[4] = go.y;
    }
    // diagonals: (5,6) = +((1,1), (-1,1)), (7,8) = -((1,1), (-1,1))
    {
        const float2 cu = make_float2(ux + uy, uy - ux), cF = make_float2(Fx + Fy, Fy - Fx);
        const float2 cZ = make_float2(Zx + Zy, Zy - Zx), cD = make_float2(dx + dy, dy - dx);
        const float w = float(D2Q9::w(5));
        collide_pair<1>(cu, cF, cZ, cD, w, mu15, muF, muZ, muD, Kf2, Bf2, pf2, omf2, Ag2, phg2, Q2,
                        omg2, make_float2(f[5], f[6]), make_float2(g[5], g[6]), fo, go);
        fv[5] = fo.x, fv[6] = fo.y, gv[5] = go.x, gv[6] = go.y;
        collide_pair<-1>(cu, cF, cZ, cD, w, mu15, muF, muZ, muD, Kf2, Bf2, pf2, omf2, Ag2, phg2, Q2,
                         omg2, make_float2(f[7], f[8]), make_float2(g[7], g[8]), fo, go);
        fv[7] = fo.x, fv[8] = fo.y, gv[7] = go.x, gv[8] = go.y;
    }
}

// One work item of the strip form: columns x0 .. x0+SW-1 (clipped to nx),
// rows ys .. ye-1 of one domain, read from level `src`, written to `dst`.
// The leading barrier also separates consecutive items of one CTA.
// TMA (tensor-tile staging, FP32 single domains): `map` is the source
// level's 3-D tensor map (x, row, slot); strips whose rows do not wrap in x
// take their population rows from it, the others copy by 16-byte chunks.
template <class T, class ST, int SW, int DEPTH, bool SLAB = false, bool TMA = false>
__device__ __forceinline__ void strip_body(const char *__restrict__ src, char *__restrict__ dst,
                                           const KP<T> &P, const int x0, const int ys,
                                           const int ye, char *smem_raw,
                                           const CUtensorMap *map = nullptr) {
    using SM = StripSmem<T, ST, SW, DEPTH>;
    using SR = typename SM::SR;
    constexpr int HP = SM::HP;
    const int t = threadIdx.x;
    const int nx = P.nx, ny = P.ny, wall = P.wall;
    const int NS = (int)P.NS;
    const int yfirst = ys - 6;

    typename SR::Desc desc;
    const int active = nx - x0 < SW ? nx - x0 : SW;
    SR::describe(desc, t, P.NS, x0 - HP, nx, active + 2 * HP);
    // the rows of this strip lie inside the level without wrapping: tiles
    const bool tma = TMA && x0 - HP >= 0 && x0 - HP + SR::LW <= nx;
    unsigned bars = 0;
    if constexpr (TMA) {
        static_assert(SM::TMA_ROWS, "TMA rows need 128-byte aligned row buffers");
        bars = smem_u32(smem_raw + SM::bar_off);
        if (tma && t == 0) {
            for (int k = 0; k < SM::NBAR; ++k) mbar_init(bars + 8 * k, 1);
            mbar_init_fence();
        }
    }
    __syncthreads();

    RingSlots<SM> R;
    auto at = [&](int off) { return smem_raw + off; };
    auto atT = [&](int off) { return reinterpret_cast<T *>(smem_raw + off); };
    // Barrier and phase parity of the rows issued for iteration it: the
    // NBAR barriers are used in turn from yfirst on, each once every NBAR
    // iterations.
    auto ibar = [&](int it) { return bars + 8u * (unsigned)((it - yfirst) % SM::NBAR); };
    auto ipar = [&](int it) { return (unsigned)((it - yfirst) / SM::NBAR) & 1u; };
    // Iteration y reads g row y+3 and f row y+1 first; both are issued
    // DEPTH iterations earlier, as one commit group.  The collisions of the
    // segment need p from row ys-1 on, so the f rows of the first warm-up
    // iterations are not loaded (the p they would give is never used).
    const int lvl_rows = SLAB ? P.rows : ny;  // rows a level holds
    auto issue_for = [&](int it, int gslot, int fslot) {
        const int gr = it + 3, fr = it + 1;
        if constexpr (TMA) {
            if (tma) {
                // one arrival announcing both rows' bytes, then the loads
                const bool g_in = gr <= ye + 2, f_in = fr >= ys - 1 && fr <= ye;
                if (t == 0 && (g_in || f_in)) {
                    const int bg = buf_row<SLAB>(P, gr), bf = buf_row<SLAB>(P, fr);
                    const bool gok = g_in && LBM_IDX_OK(P, bg >= 0 && bg < lvl_rows, 1);
                    const bool fok = f_in && LBM_IDX_OK(P, bf >= 0 && bf < lvl_rows, 1);
                    const unsigned bar = ibar(it);
                    mbar_expect_tx(bar, (gok ? SR::TMA_GB : 0u) + (fok ? SR::TMA_FB : 0u) + P.tx_extra);
                    if (gok) SR::tma_g(smem_u32(at(gslot)), map, bar, x0 - HP, bg);
                    if (fok) SR::tma_f(smem_u32(at(fslot)), map, bar, x0 - HP, bf);
                }
                return;
            }
        }
        if (gr <= ye + 2) {
            const int b = buf_row<SLAB>(P, gr);
            if (LBM_IDX_OK(P, b >= 0 && b < lvl_rows, 1)) SR::issue_g(desc, at(gslot), src, b * nx);
        }
        if (fr >= ys - 1 && fr <= ye) {
            const int b = buf_row<SLAB>(P, fr);
            if (LBM_IDX_OK(P, b >= 0 && b < lvl_rows, 1)) SR::issue_f(desc, at(fslot), src, b * nx);
        }
        cp_async_commit();  // one group per iteration, possibly empty
    };
    // Bounded wait for the rows that iteration it reads (g row it+3, and
    // f row it+1 once the segment needs it), issued for it together.
    // Every thread polls (letting one warp poll for all measured slower:
    // at the kernel's register budget the branch spills).
    auto wait_rows = [&](int it) { return mbar_wait(ibar(it), ipar(it)); };
#pragma unroll
    for (int d = 0; d < DEPTH; ++d)
        issue_for(yfirst + d, R.g[d + 3], R.f[d + SM::F1]);

    // Interior strips never wrap in x when pushing; interior rows never wrap
    // or bounce in y.
    const bool x_inner = x0 > 0 && x0 + SW < nx;
    const T c6 = T(0.5 / 3.0);
    // u, F, lap mu, grad phi of column t: c_* at row y (from the previous
    // iteration), n_* at row y+1 (computed in step 4 of this iteration)
    T c_ux = 0, c_uy = 0, c_Fx = 0, c_Fy = 0, c_lm = 0, c_gx = 0, c_gy = 0;
    T n_ux = 0, n_uy = 0, n_Fx = 0, n_Fy = 0, n_lm = 0, n_gx = 0, n_gy = 0;
    T c_f[9] = {}, n_f[9] = {};  // own f values (FCARRY): row y, row y+1

    // The row loop runs as two copies (the outer loop is unrolled, so
    // `warm` is a constant in each).  The warm-up copy (y < ys) computes
    // only what the segment's collisions read: phi from row ys-3 on, mu
    // from row ys-2 on, p from row ys-1 on (earlier rows of the rings are
    // never read), and takes no barrier before a step it skips (the
    // conditions hold for the whole CTA alike); every iteration still
    // starts with the barrier at its top.  The main copy (the segment's
    // own rows) runs every step.
    const int ymid = ys < ye ? ys : ye;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        const bool warm = pass == 0;
        for (int y = warm ? yfirst : ymid; y < (warm ? ymid : ye); ++y) {
            if (tma) {
                // g row y+3 and (once the segment needs it) f row y+1 have landed
                if (__syncthreads_or(!wait_rows(y))) {  // rows y-1 are free; or a wait ran out
                    if (t == 0 && P.err) atomicOr(P.err, 1u);
                    // wait (bounded) for the loads still in flight into this
                    // CTA's shared memory, those of iterations y+1 .. y+DEPTH-1,
                    // so that none lands after the CTA has gone
                    for (int d = 1; d < DEPTH; ++d)
                        if (y + d < ye) wait_rows(y + d);
                    return;
                }
            } else {
                cp_async_wait<DEPTH - 1>();   // g row y+3, f row y+1 have landed (own chunks)
                __syncthreads();              // ... everyone's; rows y-1 are free
            }
            issue_for(y + DEPTH, R.g[SM::NBG - 1], R.f[SM::NBF - 1]);
            const bool run_mu = !warm || y >= ys - 4, run_p = !warm || y >= ys - 2, run_col = !warm;

            // 1. phi at row y+3, columns -3 .. SW+2
            {
                const char *b = at(R.g[3]);
                T *ph = atT(R.ph[3]);
                columns<SW, 3, 3>(t, [&](int c) {
                    if (!LBM_IDX_OK(P, c >= -3 && c < SW + 3 && c + HP >= 0 && c + HP < SR::LW, 3)) return;
                    T g[9];
                    SR::read_g(b, c + HP, g);
                    ph[c] = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
                });
            }
            if (run_mu) __syncthreads();

            // 3. mu at row y+2, columns -2 .. SW+1 (Eq. 5)
            if (run_mu) {
                const int r = y + 2;
                T *mo = atT(R.mu[SM::MU0 + 2]);
                const bool ghost = wall && (r < 0 || r >= ny);
                if (!ghost) {
                    const T *pu = atT(R.ph[3]), *pc = atT(R.ph[2]), *pd = atT(R.ph[1]);
                    T *mlow = (wall && r == 0) ? atT(R.mu[SM::MU0 + 1]) : nullptr;  // row -1
                    columns<SW, 2, 1>(t, [&](int c) {
                        if (!LBM_IDX_OK(P, c >= -2 && c < SW + 2, 4)) return;
                        const T C = pc[c];
                        // lap = (2/cs2) sum w_i (phi(x + c_i) - phi(x)), differences first
                        const T ax = ((pc[c + 1] - C) + (pc[c - 1] - C)) + ((pu[c] - C) + (pd[c] - C));
                        const T dg = ((pu[c + 1] - C) + (pu[c - 1] - C)) + ((pd[c - 1] - C) + (pd[c + 1] - C));
                        const T lap = T(2.0 / 3.0) * ax + T(1.0 / 6.0) * dg;
                        const T m = P.beta4 * (C - P.phiA) * (C - P.phiB) * (C - P.phibar) - P.kappa * lap;
                        mo[c] = m;
                        if (mlow) mlow[c] = m;  // ghost row -1 mirrors row 0
                    });
                } else if (r == ny) {
                    const T *mm = atT(R.mu[SM::MU0 + 1]);  // mirror row ny-1 (already computed)
                    columns<SW, 2, 1>(t, [&](int c) { mo[c] = mm[c]; });
                }
                // r < 0 at a wall: row -1 is written when row 0 is computed;
                // rows below -1 and above ny are never read.
            }
            if (run_p) __syncthreads();

            // 4. p at row y+1, columns -1 .. SW (Eq. 32), from sum f and j of
            //    that row and phi, mu around it; thread t also keeps u, F,
            //    lap mu and grad phi of its own column t for the next
            //    iteration's collision (Eq. 31), in registers.
            if (run_p) {
                const int r = y + 1;
                T *po = atT(R.p[2]);
                if (!wall || (r >= 0 && r < ny)) {
                    const T *pu = atT(R.ph[2]), *pc = atT(R.ph[1]), *pd = atT(R.ph[0]);
                    const T *mu_ = atT(R.mu[SM::MU0 + 2]), *mc = atT(R.mu[SM::MU0 + 1]),
                            *md = atT(R.mu[SM::MU0]);
                    const char *fbr = at(R.f[SM::F1]);
                    auto point = [&](int c, bool keep) {
                        if (!LBM_IDX_OK(P, c >= -1 && c < SW + 1 && c + HP >= 0 && c + HP < SR::LW, 3)) return;
                        T f[9];
                        SR::read_f(fbr, c + HP, f);
                        const T sf = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
                        const T jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                        const T jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
                        const T phi = pc[c];
                        const T pul = pu[c - 1], pur = pu[c + 1], pdl = pd[c - 1], pdr = pd[c + 1];
                        const T gphx = T(1.0 / 3.0) * (pc[c + 1] - pc[c - 1]) +
                                       T(1.0 / 12.0) * ((pur - pul) + (pdr - pdl));
                        const T gphy = T(1.0 / 3.0) * (pu[c] - pd[c]) +
                                       T(1.0 / 12.0) * ((pur + pul) - (pdl + pdr));
                        const T M = mc[c];
                        const T mul = mu_[c - 1], mur_ = mu_[c + 1], mdl = md[c - 1], mdr = md[c + 1];
                        const T mcl = mc[c - 1], mcr = mc[c + 1], mcu = mu_[c], mcd = md[c];
                        const T gmx = T(1.0 / 3.0) * (mcr - mcl) + T(1.0 / 12.0) * ((mur_ - mul) + (mdr - mdl));
                        const T gmy = T(1.0 / 3.0) * (mcu - mcd) + T(1.0 / 12.0) * ((mur_ + mul) - (mdl + mdr));
                        const T lm = T(2.0 / 3.0) * (((mcl - M) + (mcr - M)) + ((mcu - M) + (mcd - M))) +
                                     T(1.0 / 6.0) * (((mur_ - M) + (mul - M)) + ((mdl - M) + (mdr - M)));
                        const T rho = P.rhoB + (phi - P.phiB) * P.drho;
                        const T Fx = -phi * gmx;
                        const T Fy = -phi * gmy - (rho - P.rhoref) * P.grav;
                        const T irc = T(3) * rcp_fast(rho);
                        const T ux = (jx + c6 * Fx) * irc;
                        const T uy = (jy + c6 * Fy) * irc;
                        const T udr = (ux * gphx + uy * gphy) * P.drho;
                        po[c] = sf + c6 * (udr - P.gl * rho * lm);
                        if (keep) {
                            n_ux = ux;
                            n_uy = uy;
                            n_Fx = Fx;
                            n_Fy = Fy;
                            n_lm = lm;
                            n_gx = gphx;
                            n_gy = gphy;
                            if constexpr (SM::FCARRY) {
#pragma unroll
                                for (int i = 0; i < 9; ++i) n_f[i] = f[i];
                            }
                        }
                    };
                    if constexpr (strip_threads(SW) >= SW + 2) {
                        // one pass: thread t takes column t - 1 (and collides it)
                        if (t < SW + 2) point(t - 1, t >= 1 && t <= SW);
                    } else {
                        if (t < SW) point(t, true);
                        // halo columns -1 and SW: two lanes of the last warp
                        if (t >= SW - 32 && t < SW - 30) point(t == SW - 32 ? -1 : SW, false);
                    }
                } else if (r == ny) {
                    // ghost row above the top wall: linear extrapolation of p
                    const T *p1 = atT(R.p[1]), *p2 = atT(R.p[0]);  // rows ny-1, ny-2
                    columns<SW, 1, 0>(t, [&](int c) { po[c] = T(2) * p1[c] - p2[c]; });
                }
            }
            if (run_col) __syncthreads();

            // 5. collide row y and push (Eqs. 22-29, Gamma_i = 1 + s_i): the
            //    column whose u, F, lap mu, grad phi this thread kept in step 4
            if (run_col) {
                constexpr int shift = strip_threads(SW) >= SW + 2 ? 1 : 0;
                const int c = t - shift;
                const int gx = x0 + c;
                if (c >= 0 && c < SW && gx < nx) {
                    const T *pc = atT(R.p[1]), *pu = atT(R.p[2]), *pd = atT(R.p[0]);
                    const bool lowghost = wall && y == 0;
                    const T pdm = lowghost ? T(2) * pc[c - 1] - pu[c - 1] : pd[c - 1];
                    const T pd0 = lowghost ? T(2) * pc[c] - pu[c] : pd[c];
                    const T pdp = lowghost ? T(2) * pc[c + 1] - pu[c + 1] : pd[c + 1];
                    const T gpx = T(1.0 / 3.0) * (pc[c + 1] - pc[c - 1]) +
                                  T(1.0 / 12.0) * ((pu[c + 1] - pu[c - 1]) + (pdp - pdm));
                    const T gpy = T(1.0 / 3.0) * (pu[c] - pd0) +
                                  T(1.0 / 12.0) * ((pu[c + 1] + pu[c - 1]) - (pdm + pdp));
                    const T phi = atT(R.ph[0])[c];
                    const T mu = atT(R.mu[SM::MU0])[c];
                    const T pv = pc[c];
                    const T rho = P.rhoB + (phi - P.phiB) * P.drho;
                    T f[9], g[9];
                    if constexpr (SM::FCARRY) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) f[i] = c_f[i];
                    } else {
                        SR::read_f(at(R.f[0]), c + HP, f);
                    }
                    SR::read_g(at(R.g[0]), c + HP, g);
                    T fv[9], gv[9];
                    collide(P, CellState<T>{phi, mu, pv, rho, c_ux, c_uy, c_Fx, c_Fy, c_lm, c_gx, c_gy,
                                            gpx, gpy},
                            f, g, fv, gv);
                    // pushes that neither wrap nor meet a wall (a slab's pushes
                    // across its edges land in its ghost rows)
                    const bool y_inner = (y > 0 && y < ny - 1) || (SLAB && !wall);
                    const int yl = SLAB ? y - P.y0 : y;  // row within the level
                    // deviation storage: the references of the destination
                    // cells, p and alpha mu of rows y-1 .. y+1 (cut)
                    float rP[9], rA[9];
                    if constexpr (SM::DEV) {
                        const T *mrow[3] = {atT(R.mu[SM::MU0 - 1]), atT(R.mu[SM::MU0]),
                                            atT(R.mu[SM::MU0 + 1])};
                        const T *prow[3] = {pd, pc, pu};
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
                            rP[i] = ST::ref_cut(prow[cy + 1][c + cx]);
                            rA[i] = ST::ref_cut(P.alpha * mrow[cy + 1][c + cx]);
                        }
                    }
                    // every push lands inside the level: the farthest are
                    // kb - nx - 1 and kb + nx + 1 on the fast path
                    if (x_inner && y_inner &&
                        LBM_IDX_OK(P, (yl - 1) * nx + gx - 1 >= 0 && (yl + 1) * nx + gx + 1 < lvl_rows * nx, 2)) {
                        if constexpr (SM::DEV)
                            SR::store_fast(dst, NS, nx, yl * nx + gx, fv, gv, phi, rP, rA, pv,
                                           P.alpha * mu);
                        else
                            SR::store_fast(dst, NS, nx, yl * nx + gx, fv, gv, phi);
                    } else {
                        int sl[9];
                        long long kk[9];
                        const long long k = (long long)yl * nx + gx;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const int cx = D2Q9::cx(i), cy = D2Q9::cy(i);
                            const int yd = y + cy;
                            if (wall && (yd < 0 || yd >= ny)) {
                                const T w = T(D2Q9::w(i));
                                const T cuw = T(cx) * (yd < 0 ? P.uwb : P.uwt);
                                fv[i] -= T(2) * w * rho * cuw;
                                gv[i] -= T(6) * w * phi * cuw;
                                sl[i] = D2Q9::opp(i);
                                kk[i] = k;
                                if constexpr (SM::DEV) {  // bounced back: this cell's references
                                    rP[i] = rP[0];
                                    rA[i] = rA[0];
                                }
                            } else {
                                int xd = gx + cx;
                                xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                                const int yy = SLAB ? yd - P.y0
                                                    : (yd < 0 ? yd + ny : (yd >= ny ? yd - ny : yd));
                                sl[i] = i;
                                kk[i] = (long long)yy * nx + xd;
                            }
                        }
                        bool in = true;
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            in = in && kk[i] >= 0 && kk[i] < (long long)lvl_rows * nx && sl[i] >= 0 && sl[i] < 9;
                        if (!LBM_IDX_OK(P, in, 2)) {
                        } else if constexpr (SM::DEV)
                            ST::store(dst, P.NS, sl, kk, fv, gv, phi, rP, rA, pv, P.alpha * mu);
                        else
                            ST::store(dst, P.NS, sl, kk, fv, gv, phi);
                    }
                }
            }
            c_ux = n_ux;
            c_uy = n_uy;
            c_Fx = n_Fx;
            c_Fy = n_Fy;
            c_lm = n_lm;
            c_gx = n_gx;
            c_gy = n_gy;
            if constexpr (SM::FCARRY) {
#pragma unroll
                for (int i = 0; i < 9; ++i) c_f[i] = n_f[i];
            }
            R.advance();
        }
    }
    cp_async_wait<0>();
}

// Single domain (or one y-slab of it, SLAB): CTA (bx, by) owns strip bx
// and segment by of rows ya .. yb-1.
template <class T, class ST, int SW, int DEPTH, bool SLAB>
__global__ void __launch_bounds__(strip_threads(SW), (StripSmem<T, ST, SW, DEPTH>::MINB))
k_strip(const char *__restrict__ src, char *__restrict__ dst, const __grid_constant__ KP<T> P,
        int seg_h) {
    extern __shared__ __align__(16) char smem_raw[];
    const int ys = P.ya + blockIdx.y * seg_h;
    strip_body<T, ST, SW, DEPTH, SLAB>(src, dst, P, blockIdx.x * SW, ys, min(ys + seg_h, P.yb),
                                       smem_raw);
}

// The tensor maps of one level that a storage type's row loads use.
template <int N>
struct TmaMaps {
    CUtensorMap m[N];
};

// A single domain or a y-slab with tensor-tile staging of the population
// rows (FP32 and 16-bit storage): `maps` describe the source level.
template <class T, class ST, int SW, int DEPTH, bool SLAB = false>
__global__ void __launch_bounds__(strip_threads(SW), (StripSmem<T, ST, SW, DEPTH>::MINB))
k_strip_tma(const char *__restrict__ src, char *__restrict__ dst, const __grid_constant__ KP<T> P,
            int seg_h, const __grid_constant__ TmaMaps<StripRow<ST, SW>::NMAP> maps) {
    extern __shared__ __align__(128) char smem_raw[];
    const int ys = P.ya + blockIdx.y * seg_h;
    strip_body<T, ST, SW, DEPTH, SLAB, true>(src, dst, P, blockIdx.x * SW, ys, min(ys + seg_h, P.yb),
                                             smem_raw, maps.m);
}

// ---------------------------------------------------------------- batches

// A batch advances many independent domains (each with its own size and
// parameters) with one persistent launch per strip width per step.  Work
// items are (domain, strip, segment), sorted by the host by decreasing
// cost; the CTAs claim them in that order from a ticket counter, so a CTA
// that finishes early takes the next item (longest items first, then the
// short ones fill the tail).
template <class T>
struct BatchDom {
    KP<T> kp;
    long long off[2];  // byte offsets of the domain's two levels in the state buffer
};

template <class T, class ST, int SW, int DEPTH>
__global__ void __launch_bounds__(strip_threads(SW), (StripSmem<T, ST, SW, DEPTH>::MINB))
k_strip_batch(char *__restrict__ state, const BatchDom<T> *__restrict__ doms,
              const BatchItem *__restrict__ items, int nitems, unsigned long long *__restrict__ tickets,
              int parity) {
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ KP<T> sP;
    __shared__ long long sOff[2];
    __shared__ BatchItem sW;
    __shared__ int sIt;
    // A step hands out nitems + gridDim.x tickets: ticket mod that count is
    // an item index, or (>= nitems) the one stop ticket of a CTA.  Every CTA
    // stops at its first stop ticket, so each step takes exactly that many
    // and the counter needs no reset between stream-ordered launches.
    const unsigned long long per_step = (unsigned long long)nitems + gridDim.x;
    for (;;) {
        __syncthreads();  // the previous item is done with sP, sW and sIt
        if (threadIdx.x == 0) {
            const int it = (int)(atomicAdd(tickets, 1ULL) % per_step);
            sIt = it;
            if (it < nitems) {
                const BatchItem w = items[it];
                sW = w;
                sP = doms[w.dom].kp;
                sOff[0] = doms[w.dom].off[parity];
                sOff[1] = doms[w.dom].off[1 - parity];
            }
        }
        __syncthreads();
        if (sIt >= nitems) break;
        strip_body<T, ST, SW, DEPTH>(state + sOff[0], state + sOff[1], sP, sW.x0, sW.ys, sW.ye,
                                     smem_raw);
    }
}

}  // namespace lbm
