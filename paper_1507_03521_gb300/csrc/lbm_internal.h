// lbm_internal.h — interface between the C ABI (lbm_api.cu) and the
// per-storage-type kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <cuda.h>  // CUtensorMap (type only; encoded through the runtime's driver entry point)
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <string>

#include "lbm.h"

namespace lbm {

// An NVTX range over a scope (entry points and the launches in them), for
// profilers that record NVTX (ncu --nvtx, Nsight Systems).  Without an
// attached tool a push or pop is a no-op call.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// A value set up once per device (kernel attributes, occupancy) and shared
// by every host thread that launches: the first caller on a device runs
// the set-up under a mutex and publishes the result; later callers read it.
// A failed set-up publishes nothing, so the next call tries again.
template <class V>
struct PerDevice {
    static constexpr int kMaxDev = 64;
    std::mutex mu;
    std::atomic<bool> ready[kMaxDev] = {};
    V val[kMaxDev] = {};
    // fn(dev, V &) -> cudaError_t, called with `dev` current
    template <class F>
    cudaError_t get(V &out, F &&fn) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
        if (!ready[dev].load(std::memory_order_acquire)) {
            std::lock_guard<std::mutex> lock(mu);
            if (!ready[dev].load(std::memory_order_relaxed)) {
                V v{};
                e = fn(dev, v);
                if (e != cudaSuccess) return e;
                val[dev] = v;
                ready[dev].store(true, std::memory_order_release);
            }
        }
        out = val[dev];
        return cudaSuccess;
    }
};

// Tensor maps per level at most (16-bit storage: half slots in boxes of 9
// and of 8, and the g_0 floats).
constexpr int kMaxLevelMaps = 3;

// Host-side derived parameters of one domain (FP64).
struct Derived {
    int nx, ny, wall;
    long long N, NS;  // cell count and padded slot stride
    // rows held and stepped by the strip kernel (KP in lbm_kernels.cuh):
    // the whole domain, or one y-slab of a decomposed domain
    int slab, y0, rows, ya, yb;
    int lag;  // lagged-grad-p variant (its level carries a P slot)
    // launches of this domain that run at the same time (the y-slabs of one
    // step): each strip launch sizes its grid for 1/share of the GPU
    int share = 1;
    // device word that the bounds checks of a LBM_DEBUG build set (null:
    // unchecked); release builds ignore it
    unsigned *dbg = nullptr;
    // device error word of the kernels' bounded waits (null: not reported)
    unsigned *err = nullptr;
    // test hook (lbm_test_unfinished_tiles): bytes each tile load announces
    // beyond what it brings, so that its wait runs out; 0 in normal use
    unsigned tx_extra = 0;
    // 3-D tensor maps (x, row, slot) of the two levels, for the tensor-tile
    // staging of population rows (FP32: one map per level; 16-bit storage:
    // three); tm_base[i] is the level maps tm[i] describe (null: none)
    const void *tm_base[2] = {nullptr, nullptr};
    CUtensorMap tm[2][kMaxLevelMaps];
    const CUtensorMap *map_for(const void *lvl) const {
        for (int i = 0; i < 2; ++i)
            if (tm_base[i] && tm_base[i] == lvl) return tm[i];
        return nullptr;
    }
    double phiA, phiB, phibar, rhoB, drho;
    double kappa, beta, alpha, lambda, gamma;
    double grav, rhoref, tau_f, tau_g, uwb, uwt;
};

// The 3-D tensor maps (x, row, slot) of one level of d (a whole domain or a
// y-slab) for the tensor-tile row loads of storage kind `kind` (Ops::
// tma_kind), with boxes `box` columns wide, into m[0 .. kMaxLevelMaps);
// false where the driver entry point is missing or the level cannot be
// described.
bool encode_level_maps(CUtensorMap *m, const void *lvl, const Derived &d, int kind, int box);

// Extra constants of the adjoint: derivatives of the model constants with
// respect to M and sigma.
struct AdjHost {
    double alpha1;  // alpha per unit M
    double gamma;   // gamma lambda per unit M
    double kappa1, beta1;  // kappa, beta per unit sigma
};

// Work-buffer layout of the adjoint: arrays, per-block partials, running
// (dM, dsigma) totals and the loss, then (kAdjTicketOff bytes after the
// totals) the ticket counter of the last-CTA fold.
constexpr int kAdjBlocks = 152 * 4;
constexpr size_t kAdjTicketOff = 64;
size_t adj_work_bytes(long long NS, size_t elem);
size_t adj_part_offset(long long NS, size_t elem);
size_t adj_acc_offset(long long NS, size_t elem);

// One work item of the batched strip form (see lbm_strip.cuh).
struct BatchItem {
    int dom, x0, ys, ye;
};

// Launchers of one storage type.  All are asynchronous on `s` and return
// the launch status (cudaGetLastError).
struct Ops {
    const char *name;
    size_t field_size;  // bytes of one field element (8 for FP64, else 4)
    size_t (*level_bytes)(long long NS);
    // byte offset and element size of population slot q (f_0..f_8 = 0..8,
    // g_0..g_8 = 9..17) within a level
    void (*slot_span)(long long NS, int q, size_t *off, size_t *elem);
    cudaError_t (*step)(const Derived &, const void *src, void *dst, cudaStream_t s);
    cudaError_t (*fields)(const Derived &, const void *lvl, void *phi, void *rho, void *p,
                          void *ux, void *uy, void *mu, void *P, cudaStream_t s);
    cudaError_t (*init)(const Derived &, const void *phi0, const void *ux0, const void *uy0,
                        void *lvl, cudaStream_t s);
    cudaError_t (*mass)(const Derived &, const void *lvl, double *part, int nblocks,
                        double *out2, cudaStream_t s);
    cudaError_t (*laplace)(const Derived &, const void *P, const void *phi, double xc, double yc,
                           double rin, double rout, double *part, int nblocks, double *out5,
                           cudaStream_t s);
    // batched strip form
    int strip_width;
    bool (*strip_ok)(const Derived &);
    size_t batch_dom_bytes;
    void (*batch_fill_dom)(void *host_dst, const Derived &, long long off0, long long off1);
    cudaError_t (*batch_slots)(int *slots);  // resident CTAs of one batch launch
    cudaError_t (*batch_step)(char *state, const void *doms, const BatchItem *items, int nitems,
                              unsigned long long *tickets, int parity, int grid, cudaStream_t s);
    // adjoint (plain FP64 / FP32 storage only; null otherwise)
    cudaError_t (*adj_seed)(const Derived &, const AdjHost &, const void *lvl, const void *target,
                            void *lam, void *work, cudaStream_t s);
    cudaError_t (*adj_step)(const Derived &, const AdjHost &, const void *lvl,
                            const void *lam_next, void *lam, void *work, cudaStream_t s);
    cudaError_t (*adj_init)(const Derived &, const AdjHost &, const void *phi0, const void *lam0,
                            void *phi0_bar, void *work, cudaStream_t s);
    // narrow batch kernel for strips of at most narrow_width active columns
    // (0 and null: none; every strip then runs at strip_width)
    int narrow_width;
    cudaError_t (*batch_slots_narrow)(int *slots);
    cudaError_t (*batch_step_narrow)(char *state, const void *doms, const BatchItem *items, int nitems,
                                     unsigned long long *tickets, int parity, int grid, cudaStream_t s);
    // NVTX range name of one step launch ("step <name>")
    const char *step_range = "step";
    // tensor-tile staging of population rows: the maps' box width (x
    // extent) and the level layout they describe (kTmaPlain32: 18 FP32
    // slots; kTmaHalf: g_0 floats and 17 half slots); 0 where the form does
    // not use it
    int tma_box = 0;
    int tma_kind = 0;
};
constexpr int kTmaPlain32 = 1, kTmaHalf = 2;

const Ops *ops_f64();
const Ops *ops_f32();
const Ops *ops_f16s();
const Ops *ops_bf16s();
const Ops *ops_f16d();
const Ops *ops_bf16d();
// The 16-bit deviation storage (single domains on the strip kernel only).
inline bool is_deviation_dtype(int dtype) { return dtype == LBM_F16D || dtype == LBM_BF16D; }

// Launchers for an lbm_dtype value (null if unknown).
const Ops *ops_for(int dtype);
// Parameter checks of lbm_create; empty when p is valid.
std::string check_params(const lbm_params *p);
// Derived parameters of the whole domain (Eqs. 3-4 solved, 13, 17, 33).
Derived derive(const lbm_params *p);

}  // namespace lbm

// Records a message for lbm_create_error() in the calling thread (used by
// entry points that have no handle to store it in).
void lbm_internal_set_error(const char *msg);
