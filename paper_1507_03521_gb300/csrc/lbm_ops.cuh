// lbm_ops.cuh — launchers of the kernels of lbm_kernels.cuh for one
// (compute type, storage type, tile height) choice.
#pragma once

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_adjoint.cuh"
#include "lbm_kernels.cuh"
#include "lbm_strip.cuh"
#include "lbm_strip_lag.cuh"

// Shortest segment a strip CTA marches (rows) when the one-wave grid would
// cut the strips finer.  Each segment re-reads 6 warm-up rows, but the grids
// that need segments this short are small enough to sit in L2, where the
// wider grid wins: FP32 at 512^2 ran 12.8k MLUPS with 4-row segments, 11.1k
// with 8 and 8.0k with 16 (256^2: 4.2k, 3.6k, 2.1k); from 1024^2 up the
// one-wave segments are longer than 16 rows anyway.
constexpr int kSegMinRows = 4;

// Rows per thread of the adjoint's field-and-collision tile kernel
// (k_step MODE_ADJC): 32 x 8 tiles.  On the 512^2 adjoint workload the
// backward pass took 0.317 s with them, 0.331 s with 32 x 16 tiles (512
// CTAs: 1.1 waves at 3 CTAs per SM) and 0.344-0.364 s with 32 x 32.
constexpr int kAdjRpt = 1;

namespace lbm {

template <class T>
inline KP<T> make_kp(const Derived &d) {
    KP<T> k;
    k.nx = d.nx;
    k.ny = d.ny;
    k.wall = d.wall;
    k.NS = d.NS;
    k.slab = d.slab;
    k.y0 = d.y0;
    k.rows = d.rows;
    k.ya = d.ya;
    k.yb = d.yb;
    k.phiA = T(d.phiA);
    k.phiB = T(d.phiB);
    k.phibar = T(d.phibar);
    k.rhoB = T(d.rhoB);
    k.drho = T(d.drho);
    k.kappa = T(d.kappa);
    k.beta4 = T(4.0 * d.beta);
    k.beta = T(d.beta);
    k.alpha = T(d.alpha);
    k.gl = T(d.gamma * d.lambda);
    k.grav = T(d.grav);
    k.rhoref = T(d.rhoref);
    k.itf = T(1.0 / d.tau_f);
    k.itg = T(1.0 / d.tau_g);
    k.pf = T(1.0 - 0.5 / d.tau_f);
    k.pg = T(1.0 - 0.5 / d.tau_g);
    k.uwb = T(d.uwb);
    k.uwt = T(d.uwt);
    k.err = d.err;
    k.tx_extra = d.tx_extra;
#ifdef LBM_DEBUG
    k.dbg = d.dbg;
#endif
    return k;
}

template <class T, class ST, int RPT, int SW, int DEPTH>
struct OpsImpl {
    static constexpr int TY = 8 * RPT;
    static constexpr int NT = strip_threads(SW);  // threads of a strip CTA
    using TL = Tile<T, TY>;
    using SM = StripSmem<T, ST, SW, DEPTH>;

    // The strip kernel needs 16-byte aligned rows (nx a multiple of 8) and
    // a level that 32-bit element offsets can address.
    static bool strip_ok(const Derived &d) {
        return d.nx % 8 == 0 && StripRow<ST, SW>::idx32_ok(d.NS);
    }

    struct StripCfg {
        int per_sm = 0, sms = 0;
    };
    // Opt kernel `k` in to `smem` bytes of dynamic shared memory and read
    // its resident CTAs per SM and the SM count of device `dev`.
    template <class K>
    static cudaError_t strip_cfg(K k, int smem, int dev, StripCfg &c) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, k, NT, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        return c.per_sm < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
    }

    // Opt in to the strip kernel's shared memory and size the grid to
    // one wave: strips x segments ~= resident CTAs, segments >= kSegMinRows rows.
    template <bool SLAB>
    static cudaError_t strip_grid(const Derived &d, dim3 &grid, int &seg_h) {
        static PerDevice<StripCfg> cfg;
        StripCfg c;
        cudaError_t e = cfg.get(c, [](int dev, StripCfg &v) {
            return strip_cfg(k_strip<T, ST, SW, DEPTH, SLAB>, (int)SM::bytes, dev, v);
        });
        if (e != cudaSuccess) return e;
        one_wave(d, c, grid, seg_h);
        return cudaSuccess;
    }
    // strips x segments ~= the resident CTAs c allows, segments >= kSegMinRows rows
    static void one_wave(const Derived &d, const StripCfg &c, dim3 &grid, int &seg_h) {
        const int strips = (d.nx + SW - 1) / SW;
        const int rows = d.yb - d.ya;  // rows stepped
        long long slots = (long long)c.per_sm * c.sms / (d.share > 1 ? d.share : 1);
        long long nseg = slots / strips;
        if (nseg < 1) nseg = 1;
        const long long max_seg = (rows + kSegMinRows - 1) / kSegMinRows;
        if (nseg > max_seg) nseg = max_seg;
        seg_h = (int)((rows + nseg - 1) / nseg);
        nseg = (rows + seg_h - 1) / seg_h;
        grid = dim3((unsigned)strips, (unsigned)nseg);
    }

    // The deviation storage (Store16D) runs single domains on the strip
    // kernel only: no tile-kernel step, slabs, batches or lagged variant.
    static constexpr bool kDev = IsDev<ST>::value;

    template <bool SLAB>
    static cudaError_t strip_step(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        if constexpr (kDev && SLAB) return cudaErrorNotSupported;
        else return strip_step_impl<SLAB>(d, src, dst, s);
    }
    // tensor-tile staging: single domains and y-slabs of FP32 and of raw
    // 16-bit storage on the 120-column strips (128-byte aligned row buffers)
    static constexpr bool kTmaPlain = std::is_same<ST, PlainStore<float>>::value;
    static constexpr bool kTmaHalfSt = std::is_same<ST, Store16<__half>>::value ||
                                       std::is_same<ST, Store16<__nv_bfloat16>>::value;
    static constexpr bool kTma = (kTmaPlain || kTmaHalfSt) && SM::TMA_ROWS && SW == 120;
    static constexpr int kTmaKind = kTma ? (kTmaPlain ? kTmaPlain32 : kTmaHalf) : 0;

    template <bool SLAB>
    static cudaError_t strip_step_impl(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        if constexpr (kTma) {
            if (const CUtensorMap *m = d.map_for(src)) return strip_step_tma<SLAB>(d, src, dst, m, s);
        }
        dim3 grid;
        int seg_h = 0;
        cudaError_t e = strip_grid<SLAB>(d, grid, seg_h);
        if (e != cudaSuccess) return e;
        k_strip<T, ST, SW, DEPTH, SLAB><<<grid, NT, SM::bytes, s>>>(
            static_cast<const char *>(src), static_cast<char *>(dst), make_kp<T>(d), seg_h);
        return cudaGetLastError();
    }

    template <bool SLAB>
    static cudaError_t strip_step_tma(const Derived &d, const void *src, void *dst,
                                      const CUtensorMap *m, cudaStream_t s) {
        TmaMaps<StripRow<ST, SW>::NMAP> mm;
        for (int i = 0; i < StripRow<ST, SW>::NMAP; ++i) mm.m[i] = m[i];
        static PerDevice<StripCfg> cfg;
        StripCfg c;
        cudaError_t e = cfg.get(c, [](int dev, StripCfg &v) {
            return strip_cfg(k_strip_tma<T, ST, SW, DEPTH, SLAB>, (int)SM::bytes_tma, dev, v);
        });
        if (e != cudaSuccess) return e;
        dim3 grid;
        int seg_h = 0;
        one_wave(d, c, grid, seg_h);
        k_strip_tma<T, ST, SW, DEPTH, SLAB><<<grid, NT, SM::bytes_tma, s>>>(
            static_cast<const char *>(src), static_cast<char *>(dst), make_kp<T>(d), seg_h, mm);
        return cudaGetLastError();
    }

    // The lagged-grad-p variant (strip form only; the level carries a P slot
    // after the populations).
    using LS = LagSmem<T, ST, SW, DEPTH>;
    static size_t p_offset(long long NS) { return (ST::level_bytes(NS) + 255) & ~size_t(255); }
    static cudaError_t lag_step(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        if constexpr (kDev) return cudaErrorNotSupported;
        else return lag_step_impl(d, src, dst, s);
    }
    // tensor-tile staging of the lagged variant's g and f rows (FP32)
    static constexpr bool kTmaLag = std::is_same<ST, PlainStore<float>>::value && LS::TMA_ROWS;
    // strips x segments ~= the resident CTAs c allows, segments >= 16 rows
    static void lag_grid(const Derived &d, const StripCfg &c, dim3 &grid, int &seg_h) {
        const int strips = (d.nx + SW - 1) / SW;
        long long nseg = (long long)c.per_sm * c.sms / strips;
        if (nseg < 1) nseg = 1;
        const long long max_seg = (d.ny + 15) / 16;
        if (nseg > max_seg) nseg = max_seg;
        seg_h = (int)((d.ny + nseg - 1) / nseg);
        nseg = (d.ny + seg_h - 1) / seg_h;
        grid = dim3((unsigned)strips, (unsigned)nseg);
    }
    static cudaError_t lag_step_impl(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        if constexpr (kTmaLag) {
            if (const CUtensorMap *m = d.map_for(src)) return lag_step_tma(d, src, dst, *m, s);
        }
        static PerDevice<StripCfg> cfg;
        StripCfg c;
        cudaError_t e = cfg.get(c, [](int dev, StripCfg &v) {
            return strip_cfg(k_strip_lag<T, ST, SW, DEPTH>, (int)LS::bytes, dev, v);
        });
        if (e != cudaSuccess) return e;
        dim3 grid;
        int seg_h = 0;
        lag_grid(d, c, grid, seg_h);
        k_strip_lag<T, ST, SW, DEPTH><<<grid, NT, LS::bytes, s>>>(
            static_cast<const char *>(src), static_cast<char *>(dst), make_kp<T>(d),
            (long long)p_offset(d.NS), seg_h);
        return cudaGetLastError();
    }
    static cudaError_t lag_step_tma(const Derived &d, const void *src, void *dst, const CUtensorMap &m,
                                    cudaStream_t s) {
        static PerDevice<StripCfg> cfg;
        StripCfg c;
        cudaError_t e = cfg.get(c, [](int dev, StripCfg &v) {
            return strip_cfg(k_strip_lag_tma<T, ST, SW, DEPTH>, (int)LS::bytes_tma, dev, v);
        });
        if (e != cudaSuccess) return e;
        dim3 grid;
        int seg_h = 0;
        lag_grid(d, c, grid, seg_h);
        k_strip_lag_tma<T, ST, SW, DEPTH><<<grid, NT, LS::bytes_tma, s>>>(
            static_cast<const char *>(src), static_cast<char *>(dst), make_kp<T>(d),
            (long long)p_offset(d.NS), seg_h, m);
        return cudaGetLastError();
    }

    template <int MODE, int R = RPT>
    static cudaError_t prepare() {
        // Opt in to more than 48 KB of dynamic shared memory when needed,
        // once per device.
        using TLR = Tile<T, 8 * R>;
        if (TLR::bytes <= 48 * 1024) return cudaSuccess;
        static PerDevice<int> done;
        int v = 0;
        return done.get(v, [](int, int &) {
            return cudaFuncSetAttribute(k_step<T, ST, R, MODE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TLR::bytes);
        });
    }

    static dim3 grid(const Derived &d) {
        return dim3((unsigned)((d.nx + TL::TX - 1) / TL::TX), (unsigned)((d.ny + TY - 1) / TY));
    }

    static cudaError_t step(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        // a y-slab (lbm_slabs.cu) and the lagged variant have been checked
        // for the strip form
        if constexpr (kDev) {
            if (d.lag || d.slab || !strip_ok(d)) return cudaErrorNotSupported;
            return strip_step<false>(d, src, dst, s);
        } else {
            return step_any(d, src, dst, s);
        }
    }
    static cudaError_t step_any(const Derived &d, const void *src, void *dst, cudaStream_t s) {
        if (d.lag) return strip_ok(d) ? lag_step(d, src, dst, s) : cudaErrorInvalidValue;
        if (d.slab) return strip_ok(d) ? strip_step<true>(d, src, dst, s) : cudaErrorInvalidValue;
        if (strip_ok(d)) return strip_step<false>(d, src, dst, s);
        cudaError_t e = prepare<MODE_STEP>();
        if (e != cudaSuccess) return e;
        k_step<T, ST, RPT, MODE_STEP><<<grid(d), dim3(32, 8), TL::bytes, s>>>(
            static_cast<const char *>(src), static_cast<char *>(dst), make_kp<T>(d),
            FieldOut<T>{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr});
        return cudaGetLastError();
    }

    static cudaError_t fields(const Derived &d, const void *lvl, void *phi, void *rho, void *p,
                              void *ux, void *uy, void *mu, void *P, cudaStream_t s) {
        cudaError_t e = prepare<MODE_FIELDS>();
        if (e != cudaSuccess) return e;
        FieldOut<T> o{static_cast<T *>(phi), static_cast<T *>(rho), static_cast<T *>(p),
                      static_cast<T *>(ux),  static_cast<T *>(uy),  static_cast<T *>(mu),
                      static_cast<T *>(P)};
        k_step<T, ST, RPT, MODE_FIELDS><<<grid(d), dim3(32, 8), TL::bytes, s>>>(
            static_cast<const char *>(lvl), nullptr, make_kp<T>(d), o);
        return cudaGetLastError();
    }

    static cudaError_t init(const Derived &d, const void *phi0, const void *ux0, const void *uy0,
                            void *lvl, cudaStream_t s) {
        long long nb = (d.N + 255) / 256;
        if (nb > 152 * 16) nb = 152 * 16;
        k_init<T, ST><<<(unsigned)nb, 256, 0, s>>>(
            static_cast<const T *>(phi0), static_cast<const T *>(ux0),
            static_cast<const T *>(uy0), static_cast<char *>(lvl), make_kp<T>(d));
        return cudaGetLastError();
    }

    static cudaError_t mass(const Derived &d, const void *lvl, double *part, int nblocks,
                            double *out2, cudaStream_t s) {
        k_mass_partial<T, ST><<<nblocks, 256, 0, s>>>(static_cast<const char *>(lvl),
                                                      make_kp<T>(d), part);
        k_reduce_final<<<1, 256, 0, s>>>(part, nblocks, 2, out2);
        return cudaGetLastError();
    }

    static cudaError_t laplace(const Derived &d, const void *P, const void *phi, double xc,
                               double yc, double rin, double rout, double *part, int nblocks,
                               double *out5, cudaStream_t s) {
        k_laplace_partial<T><<<nblocks, 256, 0, s>>>(static_cast<const T *>(P),
                                                     static_cast<const T *>(phi), make_kp<T>(d),
                                                     xc, yc, rin, rout, part);
        k_reduce_final<<<1, 256, 0, s>>>(part, nblocks, 5, out5);
        return cudaGetLastError();
    }

    static size_t level_bytes(long long NS) { return ST::level_bytes(NS); }

    // ---- batched strip form
    static void batch_fill_dom(void *host_dst, const Derived &d, long long off0, long long off1) {
        BatchDom<T> b;
        b.kp = make_kp<T>(d);
        b.off[0] = off0;
        b.off[1] = off1;
        *static_cast<BatchDom<T> *>(host_dst) = b;
    }

    static cudaError_t batch_slots(int *slots) {
        if constexpr (kDev) return cudaErrorNotSupported;
        else return batch_slots_impl(slots);
    }
    static cudaError_t batch_slots_impl(int *slots) {
        static PerDevice<StripCfg> cfg;
        StripCfg c;
        cudaError_t e = cfg.get(c, [](int dev, StripCfg &v) {
            return strip_cfg(k_strip_batch<T, ST, SW, DEPTH>, (int)SM::bytes, dev, v);
        });
        if (e != cudaSuccess) return e;
        *slots = c.per_sm * c.sms;
        return cudaSuccess;
    }

    static cudaError_t batch_step(char *state, const void *doms, const BatchItem *items, int nitems,
                                  unsigned long long *tickets, int parity, int grid, cudaStream_t s) {
        if constexpr (kDev) return cudaErrorNotSupported;
        else return batch_step_impl(state, doms, items, nitems, tickets, parity, grid, s);
    }
    static cudaError_t batch_step_impl(char *state, const void *doms, const BatchItem *items,
                                       int nitems, unsigned long long *tickets, int parity, int grid,
                                       cudaStream_t s) {
        int slots = 0;
        cudaError_t e = batch_slots_impl(&slots);  // also sets the shared-memory attribute
        if (e != cudaSuccess) return e;
        k_strip_batch<T, ST, SW, DEPTH><<<grid, NT, SM::bytes, s>>>(
            state, static_cast<const BatchDom<T> *>(doms), items, nitems, tickets, parity);
        return cudaGetLastError();
    }

    // ---- adjoint (plain storage only)
    static constexpr bool kPlain = std::is_same<ST, PlainStore<T>>::value;

    static AdjP<T> make_ap(const Derived &d, const AdjHost &h) {
        AdjP<T> a;
        a.k = make_kp<T>(d);
        a.alpha1 = T(h.alpha1);
        a.gamma = T(h.gamma);
        a.kappa1 = T(h.kappa1);
        a.beta1 = T(h.beta1);
        return a;
    }
    static AdjW<T> make_w(const Derived &d, void *work) {
        return AdjW<T>{static_cast<T *>(work), d.NS};
    }
    static int adj_grid(const Derived &d) {
        long long nb = (d.N + 255) / 256;
        return (int)(nb < kAdjBlocks ? nb : kAdjBlocks);
    }
    static double *part(const Derived &d, void *work) {
        return reinterpret_cast<double *>(static_cast<char *>(work) +
                                          adj_part_offset(d.NS, sizeof(T)));
    }
    static double *acc(const Derived &d, void *work) {
        return reinterpret_cast<double *>(static_cast<char *>(work) +
                                          adj_acc_offset(d.NS, sizeof(T)));
    }
    // ticket counter of k_adj_muphi's last-CTA fold, after the totals
    static unsigned *ticket(const Derived &d, void *work) {
        return reinterpret_cast<unsigned *>(static_cast<char *>(work) +
                                            adj_acc_offset(d.NS, sizeof(T)) + kAdjTicketOff);
    }

    static cudaError_t adj_seed(const Derived &d, const AdjHost &h, const void *lvl,
                                const void *target, void *lam, void *work, cudaStream_t s) {
        const int nb = adj_grid(d);
        k_adj_seed<T><<<nb, 256, 0, s>>>(static_cast<const T *>(lvl), static_cast<const T *>(target),
                                         static_cast<T *>(lam), make_ap(d, h), part(d, work));
        k_reduce_final<<<1, 256, 0, s>>>(part(d, work), nb, 1, acc(d, work) + 2);
        return cudaGetLastError();
    }

    static cudaError_t adj_step(const Derived &d, const AdjHost &h, const void *lvl,
                                const void *lam_next, void *lam, void *work, cudaStream_t s) {
        const AdjP<T> P = make_ap(d, h);
        const AdjW<T> W = make_w(d, work);
        const int nb = adj_grid(d);
        T *L = static_cast<T *>(lam);
        // the forward fields of step t and the collision adjoint, in one
        // tile-kernel launch (rows per thread RA)
        constexpr int RA = kAdjRpt;
        using TLA = Tile<T, 8 * RA>;
        cudaError_t e = prepare<MODE_ADJC, RA>();
        if (e != cudaSuccess) return e;
        FieldOut<T> fo{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        fo.adj = W.a;
        fo.adj_ns = d.NS;
        fo.beta1x4 = T(4) * P.beta1;
        fo.kappa1 = P.kappa1;
        fo.lam_next = static_cast<const T *>(lam_next);
        fo.lam = L;
        const dim3 ga((unsigned)((d.nx + TLA::TX - 1) / TLA::TX), (unsigned)((d.ny + 8 * RA - 1) / (8 * RA)));
        k_step<T, ST, RA, MODE_ADJC><<<ga, dim3(32, 8), TLA::bytes, s>>>(
            static_cast<const char *>(lvl), nullptr, make_kp<T>(d), fo);
        k_adj_p<T><<<nb, 256, 0, s>>>(L, P, W);
        // mu and phi adjoints, with the (M, sigma) sums folded by the last CTA
        const long long tiles = (long long)((d.nx + kMpTX - 1) / kMpTX) * ((d.ny + kMpTY - 1) / kMpTY);
        const int nt = (int)(tiles < kAdjBlocks ? tiles : kAdjBlocks);
        k_adj_muphi<T><<<nt, 256, 0, s>>>(L, P, W, part(d, work), acc(d, work), ticket(d, work));
        return cudaGetLastError();
    }

    static cudaError_t adj_init(const Derived &d, const AdjHost &h, const void *phi0,
                                const void *lam0, void *phi0_bar, void *work, cudaStream_t s) {
        const AdjP<T> P = make_ap(d, h);
        const AdjW<T> W = make_w(d, work);
        const int nb = adj_grid(d);
        k_adj_phi0<T><<<nb, 256, 0, s>>>(static_cast<const T *>(phi0), P, W);
        k_adj_f1<T><<<nb, 256, 0, s>>>(P, W);
        k_adj_init_a<T><<<nb, 256, 0, s>>>(static_cast<const T *>(lam0), P, W);
        k_adj_init_b<T><<<nb, 256, 0, s>>>(static_cast<const T *>(lam0), static_cast<T *>(phi0_bar),
                                           P, W);
        k_adj_theta<T><<<nb, 256, 0, s>>>(P, W, part(d, work));
        k_adj_accumulate<<<1, 256, 0, s>>>(part(d, work), nb, 2, acc(d, work));
        return cudaGetLastError();
    }

    static constexpr int kSW = SW;

    // The launcher table; the batched form's launchers come from B, which
    // may be this type at another strip width.
    template <class B, class BN = void>
    static Ops table(const char *name) {
        Ops o{name,        sizeof(T),   &level_bytes, &ST::slot_span,
              &step,       &fields,     &init,        &mass,
              &laplace,    B::kSW,      &strip_ok,    sizeof(BatchDom<T>),
              &B::batch_fill_dom,       &B::batch_slots,   &B::batch_step,
              kPlain ? &adj_seed : nullptr, kPlain ? &adj_step : nullptr,
              kPlain ? &adj_init : nullptr, 0, nullptr, nullptr};
        static const std::string range = std::string("step ") + name;
        o.step_range = range.c_str();
        o.tma_box = kTma ? SM::LW : 0;
        o.tma_kind = kTmaKind;
        if constexpr (!std::is_same<BN, void>::value) {
            o.narrow_width = BN::kSW;
            o.batch_slots_narrow = &BN::batch_slots;
            o.batch_step_narrow = &BN::batch_step;
        }
        return o;
    }
    static const Ops *ops(const char *name) {
        static const Ops o = table<OpsImpl>(name);
        return &o;
    }
    // Single domains and slabs at this strip width, batches at B's, and the
    // batches' remainder strips of at most BN's width at BN's.  The batch's
    // domains have widths that are multiples of 32, which whole-warp strips
    // tile exactly; a strip width chosen for single pass per step (not a
    // multiple of 32) would leave a narrow remainder strip in most of them.
    // A remainder of 64 columns or fewer on a 128-column CTA would leave
    // half its threads or more idle: BN's CTAs are sized to it.
    template <class B, class BN = void>
    static const Ops *ops_batch_from(const char *name) {
        static const Ops o = table<B, BN>(name);
        return &o;
    }
};

}  // namespace lbm
