// lbm_api.cu — the C ABI declared in include/lbm.h.
//
// Host-side bookkeeping only: parameter validation and derivation (Eqs. 3-4
// solved for kappa and beta, Eq. 13, Eq. 17, Eq. 33), buffer layout, and
// the launch sequence of each entry point.  Every step of the method runs
// in the kernels of lbm_kernels.cuh.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

using lbm::Derived;
using lbm::Ops;

namespace {

constexpr int kPartBlocks = 152 * 4;  // reduction grid: 4 CTAs per SM
constexpr int kFieldSlots = 7;        // phi, rho, p, ux, uy, mu, P

thread_local std::string g_create_err;

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
    size_t level, state, field_slot, part_off, out_off, work;
};

// The lagged variant's P slot follows the populations of a level.
size_t p_slot_offset(const Derived &d, const Ops *ops) { return round256(ops->level_bytes(d.NS)); }

// Bytes of one time level as get/set_state copy it.
size_t level_state_bytes(const Derived &d, const Ops *ops) {
    return d.lag ? p_slot_offset(d, ops) + (size_t)d.NS * ops->field_size : ops->level_bytes(d.NS);
}

Layout layout(const Derived &d, const Ops *ops) {
    Layout L;
    L.level = round256(level_state_bytes(d, ops));
    L.state = 2 * L.level;
    L.field_slot = round256((size_t)d.NS * ops->field_size);
    L.part_off = kFieldSlots * L.field_slot;
    L.out_off = L.part_off + round256((size_t)kPartBlocks * 5 * sizeof(double));
    L.work = L.out_off + 256;
    return L;
}

}  // namespace

void lbm_internal_set_error(const char *msg) { g_create_err = msg ? msg : ""; }

namespace lbm {

const Ops *ops_for(int dtype) {
    switch (dtype) {
        case LBM_F64: return lbm::ops_f64();
        case LBM_F32: return lbm::ops_f32();
        case LBM_F16S: return lbm::ops_f16s();
        case LBM_BF16S: return lbm::ops_bf16s();
        case LBM_F16D: return lbm::ops_f16d();
        case LBM_BF16D: return lbm::ops_bf16d();
        default: return nullptr;
    }
}

// Parameter checks; returns an empty string when prm is valid.
std::string check_params(const lbm_params *p) {
    if (!p) return "null parameter block";
    if (p->nx < 5 || p->ny < 5) return "nx and ny must be >= 5";
    if ((long long)p->nx * p->ny > (1LL << 34)) return "grid too large";
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return "tau_f and tau_g must exceed 1/2";
    if (!(p->rho_A > 0.0) || !(p->rho_B > 0.0)) return "rho_A and rho_B must be positive";
    if (!(p->W > 0.0)) return "W must be positive";
    if (!(p->sigma >= 0.0) || !(p->M >= 0.0)) return "sigma and M must be non-negative";
    if (!(p->phi_A != p->phi_B)) return "phi_A and phi_B must differ";
    if (p->rho_B * p->phi_A - p->rho_A * p->phi_B == 0.0) return "gamma undefined for these rho, phi";
    if (p->bc_x != LBM_PERIODIC) return "bc_x must be LBM_PERIODIC";
    if (p->bc_y != LBM_PERIODIC && p->bc_y != LBM_WALL) return "bc_y must be LBM_PERIODIC or LBM_WALL";
    if (!ops_for(p->dtype)) return "unknown dtype";
    if (p->gradp_lag != 0 && p->gradp_lag != 1) return "gradp_lag must be 0 or 1";
    if (p->gradp_lag && p->nx % 8 != 0) return "the lagged-grad-p variant needs nx a multiple of 8";
    if (is_deviation_dtype(p->dtype) && p->nx % 8 != 0)
        return "the deviation storage (LBM_F16D, LBM_BF16D) needs nx a multiple of 8";
    if (is_deviation_dtype(p->dtype) && p->gradp_lag)
        return "the deviation storage takes the synchronous step (gradp_lag = 0)";
    const double vals[] = {p->rho_A, p->rho_B, p->phi_A, p->phi_B, p->sigma, p->W, p->M,
                           p->tau_f, p->tau_g, p->gravity, p->rho_ref, p->u_wall_bottom,
                           p->u_wall_top};
    for (double v : vals)
        if (!std::isfinite(v)) return "non-finite parameter";
    return "";
}

Derived derive(const lbm_params *p) {
    Derived d;
    d.nx = p->nx;
    d.ny = p->ny;
    d.wall = p->bc_y == LBM_WALL;
    d.N = (long long)p->nx * p->ny;
    d.NS = (d.N + 127) / 128 * 128;
    d.slab = 0;
    d.y0 = 0;
    d.rows = d.ny;
    d.ya = 0;
    d.yb = d.ny;
    d.lag = p->gradp_lag ? 1 : 0;
    const double dphi = p->phi_A - p->phi_B;
    d.phiA = p->phi_A;
    d.phiB = p->phi_B;
    d.phibar = 0.5 * (p->phi_A + p->phi_B);
    d.rhoB = p->rho_B;
    d.drho = (p->rho_A - p->rho_B) / dphi;                    // Eq. 13
    d.kappa = 3.0 * p->sigma * p->W / (2.0 * dphi * dphi);    // Eqs. 3-4
    d.beta = 12.0 * p->sigma / (p->W * dphi * dphi * dphi * dphi);
    d.lambda = p->M;
    d.alpha = p->M / ((p->tau_g - 0.5) / 3.0);                // Eq. 33
    d.gamma = (p->rho_A - p->rho_B) / (p->rho_B * p->phi_A - p->rho_A * p->phi_B);  // Eq. 17
    d.grav = p->gravity;
    d.rhoref = p->rho_ref;
    d.tau_f = p->tau_f;
    d.tau_g = p->tau_g;
    d.uwb = d.wall ? p->u_wall_bottom : 0.0;
    d.uwt = d.wall ? p->u_wall_top : 0.0;
    return d;
}

}  // namespace lbm

using lbm::check_params;
using lbm::derive;
using lbm::ops_for;

namespace lbm {
// Adjoint work buffer: A_COUNT field arrays of NS elements, then the
// per-block partials, then 4 doubles (dM, dsigma totals, loss, spare).
constexpr int kAdjArrays = 36;
size_t adj_part_offset(long long NS, size_t elem) {
    return round256((size_t)kAdjArrays * (size_t)NS * elem);
}
size_t adj_acc_offset(long long NS, size_t elem) {
    return adj_part_offset(NS, elem) + round256((size_t)kAdjBlocks * 2 * sizeof(double));
}
size_t adj_work_bytes(long long NS, size_t elem) { return adj_acc_offset(NS, elem) + 256; }
}  // namespace lbm

struct lbm_sim {
    lbm_params prm;
    Derived d;
    const Ops *ops;
    Layout L;
    cudaStream_t stream;
    char *state = nullptr;
    char *work = nullptr;
    int cur = 0;  // index of the level holding the current time
    int64_t steps = 0;
    bool initialized = false;
    std::string err;
    // adjoint segments (lbm_adj_segment): optional CUDA-graph replay of the
    // launch sequence, kept for the last (n, buffers) it was captured for
    bool adj_graph = false;
    cudaGraphExec_t adj_exec = nullptr;
    int64_t adj_n = -1;
    size_t adj_stride = 0;
    const void *adj_key[4] = {nullptr, nullptr, nullptr, nullptr};
    // overlapped reverse sweep (lbm_adj_reverse_overlap): the second stream
    // that recomputes the next segment, fork/join events, and the graphs of
    // the last two calls (a sweep alternates two state buffers)
    cudaStream_t adj_side = nullptr;
    cudaEvent_t adj_fork = nullptr, adj_join = nullptr;
    struct OvGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t n = -1, n_next = -1;
        size_t stride = 0;
        const void *key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    } adj_ov[2];
    int adj_ov_next = 0;  // entry the next capture replaces

    ~lbm_sim() {
        if (adj_exec) cudaGraphExecDestroy(adj_exec);
        for (auto &g : adj_ov)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (adj_fork) cudaEventDestroy(adj_fork);
        if (adj_join) cudaEventDestroy(adj_join);
        if (adj_side) cudaStreamDestroy(adj_side);
    }

    char *level(int i) { return state + (size_t)i * L.level; }
    char *slot(int i) { return work + (size_t)i * L.field_slot; }
    double *part() { return reinterpret_cast<double *>(work + L.part_off); }
    double *out() { return reinterpret_cast<double *>(work + L.out_off); }

    lbm_status fail(lbm_status s, const std::string &m) {
        err = m;
        return s;
    }
    lbm_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return LBM_OK;
        err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
        return LBM_ERR_CUDA;
    }
    lbm_status ready() {
        if (!state || !work) return fail(LBM_ERR_STATE, "buffers not bound");
        return LBM_OK;
    }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The 3-D tensor map (x, row, slot) of one FP32 level for the tensor-tile
// staging: box = `box` columns x 1 row x 9 slots (one f or g row), no
// swizzle, zero fill outside (never read: only strips whose rows lie inside
// the level use the map).  False when the map cannot be made; the strip
// kernel then copies by chunks.
namespace lbm {
// One 3-D map (x, row, slot) of `nslots` slots of `elem`-byte elements,
// slot s at byte offset s * slot_stride from base; boxes box x 1 x bslots.
static bool encode_map(CUtensorMap *m, CUtensorMapDataType type, const void *base, int nx, int rows,
                       int nslots, int elem, size_t slot_stride, int box, int bslots) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || box <= 0 || box > 256 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)rows, (cuuint64_t)nslots};
    cuuint64_t strides[2] = {(cuuint64_t)nx * elem, (cuuint64_t)slot_stride};
    cuuint32_t boxd[3] = {(cuuint32_t)box, 1, (cuuint32_t)bslots};
    cuuint32_t estr[3] = {1, 1, 1};
    if (((strides[0] | strides[1]) & 15) || ((size_t)box * elem) % 16) return false;
    return enc(m, type, 3, const_cast<void *>(base), dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_level_maps(CUtensorMap *m, const void *lvl, const Derived &d, int kind, int box) {
    // rows a level holds: the domain's, or a y-slab's own rows and ghosts
    const int rows = d.slab ? d.rows : d.ny;
    const char *b = static_cast<const char *>(lvl);
    if (kind == kTmaPlain32)  // f_0..f_8, g_0..g_8 as FP32 slots NS apart
        return encode_map(&m[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, b, d.nx, rows, 18, 4,
                          (size_t)d.NS * 4, box, 9);
    if (kind == kTmaHalf)  // g_0 as NS floats, then 17 half slots NS apart
        return encode_map(&m[0], CU_TENSOR_MAP_DATA_TYPE_UINT16, b + (size_t)d.NS * 4, d.nx, rows, 17, 2,
                          (size_t)d.NS * 2, box, 9) &&
               encode_map(&m[1], CU_TENSOR_MAP_DATA_TYPE_UINT16, b + (size_t)d.NS * 4, d.nx, rows, 17, 2,
                          (size_t)d.NS * 2, box, 8) &&
               encode_map(&m[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, b, d.nx, rows, 1, 4, (size_t)d.NS * 4,
                          box, 1);
    return false;
}
}  // namespace lbm
using lbm::encode_level_maps;

// The kernels' error word: bit 0, a bounded wait for a tile load ran out.
static lbm_status error_word(lbm_sim *s) {
    unsigned w = 0;
    if (cudaMemcpy(&w, s->d.err, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
        return s->fail(LBM_ERR_CUDA, "reading the kernels' error word");
    if (w & 1u) return s->fail(LBM_ERR_TIMEOUT, "a bounded wait for a tile load ran out");
    return LBM_OK;
}

// LBM_DEBUG builds: the bounds-check word, read after the stream is
// synchronised; a set bit is a failed index check (code = bit number).
static lbm_status debug_word(lbm_sim *s) {
#ifdef LBM_DEBUG
    unsigned w = 0;
    if (cudaMemcpy(&w, s->d.dbg, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
        return s->fail(LBM_ERR_CUDA, "reading the LBM_DEBUG check word");
    if (w) return s->fail(LBM_ERR_STATE, "LBM_DEBUG index check failed, codes 0x" + [&] {
        char b[16];
        snprintf(b, sizeof(b), "%x", w);
        return std::string(b);
    }());
#else
    (void)s;
#endif
    return LBM_OK;
}

#define LBM_CK(sim, call)                                   \
    do {                                                    \
        lbm_status st__ = (sim)->cuda((call), #call);       \
        if (st__ != LBM_OK) return st__;                    \
    } while (0)

extern "C" {

int lbm_version(void) { return 1; }

lbm_status lbm_buffer_sizes(const lbm_params *prm, size_t *state_bytes, size_t *work_bytes) {
    std::string m = check_params(prm);
    if (!m.empty()) {
        g_create_err = m;
        return LBM_ERR_ARG;
    }
    const Derived d = derive(prm);
    const Layout L = layout(d, ops_for(prm->dtype));
    if (state_bytes) *state_bytes = L.state;
    if (work_bytes) *work_bytes = L.work;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params *prm, void *stream, lbm_sim **out) {
    if (!out) {
        g_create_err = "null output pointer";
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    std::string m = check_params(prm);
    if (!m.empty()) {
        g_create_err = m;
        return LBM_ERR_ARG;
    }
    lbm_sim *s = new (std::nothrow) lbm_sim();
    if (!s) {
        g_create_err = "host allocation failed";
        return LBM_ERR_NOMEM;
    }
    s->prm = *prm;
    s->d = derive(prm);
    s->ops = ops_for(prm->dtype);
    if ((s->d.lag || lbm::is_deviation_dtype(prm->dtype)) && !s->ops->strip_ok(s->d)) {
        delete s;
        g_create_err = "this dtype or variant needs the strip form (grid too large)";
        return LBM_ERR_ARG;
    }
    s->L = layout(s->d, s->ops);
    s->stream = static_cast<cudaStream_t>(stream);
    g_create_err.clear();
    *out = s;
    return LBM_OK;
}

lbm_status lbm_bind_buffers(lbm_sim *s, void *state, size_t state_bytes, void *work,
                            size_t work_bytes) {
    if (!s) return LBM_ERR_ARG;
    if (!state || !work) return s->fail(LBM_ERR_ARG, "null buffer");
    if ((reinterpret_cast<uintptr_t>(state) & 255) || (reinterpret_cast<uintptr_t>(work) & 255))
        return s->fail(LBM_ERR_ARG, "buffers must be 256-byte aligned");
    if (state_bytes < s->L.state || work_bytes < s->L.work)
        return s->fail(LBM_ERR_NOMEM, "bound buffer smaller than lbm_buffer_sizes");
    s->state = static_cast<char *>(state);
    s->work = static_cast<char *>(work);
    s->initialized = false;
    // the bounds-check word of LBM_DEBUG builds and the kernels' error
    // word: spare words of the reduction output area
    s->d.dbg = reinterpret_cast<unsigned *>(s->work + s->L.out_off + 128);
    s->d.err = reinterpret_cast<unsigned *>(s->work + s->L.out_off + 132);
    // tensor maps of the two levels for the tensor-tile staging
    s->d.tm_base[0] = s->d.tm_base[1] = nullptr;
    if (s->ops->tma_kind > 0 && s->ops->strip_ok(s->d))
        for (int i = 0; i < 2; ++i)
            if (encode_level_maps(s->d.tm[i], s->level(i), s->d, s->ops->tma_kind, s->ops->tma_box))
                s->d.tm_base[i] = s->level(i);
    return LBM_OK;
}

lbm_status lbm_init_phi(lbm_sim *s, const void *phi, const void *ux, const void *uy, int on_host) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_init_phi");
    if (lbm_status st = s->ready()) return st;
    if (!phi) return s->fail(LBM_ERR_ARG, "phi is null");
    const size_t fb = (size_t)s->d.N * s->ops->field_size;
    const void *dphi = phi, *dux = ux, *duy = uy;
    if (on_host) {
        LBM_CK(s, cudaMemcpyAsync(s->slot(0), phi, fb, cudaMemcpyHostToDevice, s->stream));
        dphi = s->slot(0);
        if (ux) {
            LBM_CK(s, cudaMemcpyAsync(s->slot(3), ux, fb, cudaMemcpyHostToDevice, s->stream));
            dux = s->slot(3);
        }
        if (uy) {
            LBM_CK(s, cudaMemcpyAsync(s->slot(4), uy, fb, cudaMemcpyHostToDevice, s->stream));
            duy = s->slot(4);
        }
    }
    s->cur = 0;
    LBM_CK(s, cudaMemsetAsync(s->d.dbg, 0, 2 * sizeof(unsigned), s->stream));  // dbg, err
    LBM_CK(s, s->ops->init(s->d, dphi, dux, duy, s->level(0), s->stream));
    if (s->d.lag)  // the previous-step pressure of the initial state: p = 0
        LBM_CK(s, cudaMemsetAsync(s->level(0) + p_slot_offset(s->d, s->ops), 0,
                                  (size_t)s->d.NS * s->ops->field_size, s->stream));
    if (on_host) LBM_CK(s, cudaStreamSynchronize(s->stream));
    s->steps = 0;
    s->initialized = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_sim *s, int64_t n) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_step");
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_step before lbm_init_phi");
    if (n < 0) return s->fail(LBM_ERR_ARG, "negative step count");
    for (int64_t t = 0; t < n; ++t) {
        lbm::NvtxRange r_launch(s->ops->step_range);
        LBM_CK(s, s->ops->step(s->d, s->level(s->cur), s->level(1 - s->cur), s->stream));
        s->cur = 1 - s->cur;
        s->steps++;
    }
    return LBM_OK;
}

lbm_status lbm_fields(lbm_sim *s, void *phi, void *rho, void *p, void *ux, void *uy, void *mu,
                      int on_host) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_fields");
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_fields before lbm_init_phi");
    void *user[6] = {phi, rho, p, ux, uy, mu};
    void *dev[6];
    for (int i = 0; i < 6; ++i) dev[i] = on_host ? (user[i] ? s->slot(i) : nullptr) : user[i];
    LBM_CK(s, s->ops->fields(s->d, s->level(s->cur), dev[0], dev[1], dev[2], dev[3], dev[4],
                             dev[5], nullptr, s->stream));
    if (on_host) {
        const size_t fb = (size_t)s->d.N * s->ops->field_size;
        for (int i = 0; i < 6; ++i)
            if (user[i])
                LBM_CK(s, cudaMemcpyAsync(user[i], dev[i], fb, cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(s, cudaStreamSynchronize(s->stream));
    }
    return LBM_OK;
}

lbm_status lbm_mass(lbm_sim *s, double *mass, double *phi_total) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_mass");
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_mass before lbm_init_phi");
    long long nb = (s->d.N + 255) / 256;
    const int nblocks = (int)(nb < kPartBlocks ? nb : kPartBlocks);
    double h[2];
    LBM_CK(s, s->ops->mass(s->d, s->level(s->cur), s->part(), nblocks, s->out(), s->stream));
    LBM_CK(s, cudaMemcpyAsync(h, s->out(), sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    if (lbm_status st = error_word(s)) return st;
    if (lbm_status st = debug_word(s)) return st;
    if (mass) *mass = h[0];
    if (phi_total) *phi_total = h[1];
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
        return s->fail(LBM_ERR_NONFINITE, "non-finite mass or phi total");
    return LBM_OK;
}

lbm_status lbm_laplace(lbm_sim *s, double xc, double yc, double R, double *dP, double *R_eff) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_laplace");
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_laplace before lbm_init_phi");
    LBM_CK(s, s->ops->fields(s->d, s->level(s->cur), s->slot(0), nullptr, nullptr, nullptr,
                             nullptr, nullptr, s->slot(6), s->stream));
    long long nb = (s->d.N + 255) / 256;
    const int nblocks = (int)(nb < kPartBlocks ? nb : kPartBlocks);
    const double W = s->prm.W;
    double h[5];
    LBM_CK(s, s->ops->laplace(s->d, s->slot(6), s->slot(0), xc, yc, R - 2.0 * W, R + 2.0 * W,
                              s->part(), nblocks, s->out(), s->stream));
    LBM_CK(s, cudaMemcpyAsync(h, s->out(), sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    if (lbm_status st = error_word(s)) return st;
    if (lbm_status st = debug_word(s)) return st;
    if (dP) *dP = (h[1] > 0 && h[3] > 0) ? h[0] / h[1] - h[2] / h[3] : NAN;
    if (R_eff) *R_eff = std::sqrt(h[4] / 3.14159265358979323846);
    if (!std::isfinite(h[0]) || !std::isfinite(h[2]) || !std::isfinite(h[4]))
        return s->fail(LBM_ERR_NONFINITE, "non-finite pressure or phi");
    return LBM_OK;
}

size_t lbm_state_bytes(const lbm_sim *s) { return s ? level_state_bytes(s->d, s->ops) : 0; }

lbm_status lbm_get_state(lbm_sim *s, void *dst, int on_host, int64_t *step) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_get_state before lbm_init_phi");
    if (!dst) return s->fail(LBM_ERR_ARG, "null destination");
    LBM_CK(s, cudaMemcpyAsync(dst, s->level(s->cur), lbm_state_bytes(s),
                              on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                              s->stream));
    if (on_host) LBM_CK(s, cudaStreamSynchronize(s->stream));
    if (step) *step = s->steps;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_sim *s, const void *src, int on_host, int64_t step) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!src) return s->fail(LBM_ERR_ARG, "null source");
    s->cur = 0;
    LBM_CK(s, cudaMemsetAsync(s->d.dbg, 0, 2 * sizeof(unsigned), s->stream));  // dbg, err
    LBM_CK(s, cudaMemcpyAsync(s->level(0), src, lbm_state_bytes(s),
                              on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              s->stream));
    if (on_host) LBM_CK(s, cudaStreamSynchronize(s->stream));
    s->steps = step;
    s->initialized = true;
    return LBM_OK;
}

int64_t lbm_step_count(const lbm_sim *s) { return s ? s->steps : 0; }

const char *lbm_last_error(const lbm_sim *s) { return s ? s->err.c_str() : "null handle"; }

const char *lbm_create_error(void) { return g_create_err.c_str(); }

void lbm_destroy(lbm_sim *s) { delete s; }

// ------------------------------------------------------------- adjoint

static lbm::AdjHost adj_host(const lbm_params &p) {
    lbm::AdjHost h;
    const double d = p.phi_A - p.phi_B;
    h.alpha1 = 1.0 / ((p.tau_g - 0.5) / 3.0);
    h.gamma = (p.rho_A - p.rho_B) / (p.rho_B * p.phi_A - p.rho_A * p.phi_B);
    h.kappa1 = 3.0 * p.W / (2.0 * d * d);
    h.beta1 = 12.0 / (p.W * d * d * d * d);
    return h;
}

static lbm_status adj_ready(lbm_sim *s, const void *work) {
    if (!s) return LBM_ERR_ARG;
    if (!s->ops->adj_step) return s->fail(LBM_ERR_ARG, "the adjoint needs LBM_F64 or LBM_F32");
    if (s->d.lag) return s->fail(LBM_ERR_ARG, "the adjoint is of the synchronous step (gradp_lag = 0)");
    if (!work) return s->fail(LBM_ERR_ARG, "null adjoint work buffer");
    if (reinterpret_cast<uintptr_t>(work) & 255)
        return s->fail(LBM_ERR_ARG, "adjoint work buffer must be 256-byte aligned");
    return LBM_OK;
}

lbm_status lbm_adj_work_bytes(const lbm_sim *s, size_t *bytes) {
    if (!s || !bytes) return LBM_ERR_ARG;
    if (!s->ops->adj_step || s->d.lag) return LBM_ERR_ARG;
    *bytes = lbm::adj_work_bytes(s->d.NS, s->ops->field_size);
    return LBM_OK;
}

lbm_status lbm_adj_reset(lbm_sim *s, void *work) {
    if (lbm_status st = adj_ready(s, work)) return st;
    char *acc = static_cast<char *>(work) + lbm::adj_acc_offset(s->d.NS, s->ops->field_size);
    LBM_CK(s, cudaMemsetAsync(acc, 0, lbm::kAdjTicketOff + sizeof(unsigned), s->stream));
    return LBM_OK;
}

lbm_status lbm_adj_seed(lbm_sim *s, const void *state_T, const void *phi_target, void *lam_T,
                        void *work, double *loss) {
    if (lbm_status st = adj_ready(s, work)) return st;
    if (!state_T || !phi_target || !lam_T) return s->fail(LBM_ERR_ARG, "null pointer");
    LBM_CK(s, s->ops->adj_seed(s->d, adj_host(s->prm), state_T, phi_target, lam_T, work, s->stream));
    if (loss) {
        const char *acc = static_cast<const char *>(work) + lbm::adj_acc_offset(s->d.NS, s->ops->field_size);
        LBM_CK(s, cudaMemcpyAsync(loss, acc + 2 * sizeof(double), sizeof(double),
                                  cudaMemcpyDeviceToHost, s->stream));
        LBM_CK(s, cudaStreamSynchronize(s->stream));
    }
    return LBM_OK;
}

lbm_status lbm_adj_step(lbm_sim *s, const void *state_t, const void *lam_next, void *lam_t,
                        void *work) {
    lbm::NvtxRange r_call("lbm_adj_step");
    if (lbm_status st = adj_ready(s, work)) return st;
    if (!state_t || !lam_next || !lam_t) return s->fail(LBM_ERR_ARG, "null pointer");
    if (lam_next == lam_t) return s->fail(LBM_ERR_ARG, "lam_next and lam_t must differ");
    LBM_CK(s, s->ops->adj_step(s->d, adj_host(s->prm), state_t, lam_next, lam_t, work, s->stream));
    return LBM_OK;
}

lbm_status lbm_adj_init(lbm_sim *s, const void *phi0, const void *lam_0, void *phi0_bar,
                        void *work) {
    if (lbm_status st = adj_ready(s, work)) return st;
    if (!phi0 || !lam_0 || !phi0_bar) return s->fail(LBM_ERR_ARG, "null pointer");
    LBM_CK(s, s->ops->adj_init(s->d, adj_host(s->prm), phi0, lam_0, phi0_bar, work, s->stream));
    return LBM_OK;
}

lbm_status lbm_test_unfinished_tiles(lbm_sim *s, int on) {
    if (!s) return LBM_ERR_ARG;
    s->d.tx_extra = on ? 16u : 0u;
    return LBM_OK;
}

lbm_status lbm_adj_set_graph(lbm_sim *s, int on) {
    if (!s) return LBM_ERR_ARG;
    if (on && (s->stream == nullptr || s->stream == cudaStreamLegacy || s->stream == cudaStreamPerThread))
        return s->fail(LBM_ERR_ARG, "graph replay needs a stream other than the default stream");
    s->adj_graph = on != 0;
    return LBM_OK;
}

// The recompute of one segment on stream st: n - 1 forward steps that fill
// levels 1 .. n-1 of `states` from level 0.  It runs the kernel lbm_step
// runs: where the handle's levels have tensor maps (FP32), each source level
// of the segment gets one too.
static cudaError_t adj_recompute_issue(lbm_sim *s, int64_t n, char *states, size_t lb,
                                       cudaStream_t st) {
    const Ops *o = s->ops;
    Derived dk = s->d;
    for (int64_t k = 1; k < n; ++k) {
        char *src = states + (k - 1) * lb;
        dk.tm_base[0] = dk.tm_base[1] = nullptr;
        if (s->d.tm_base[0] && encode_level_maps(dk.tm[0], src, dk, o->tma_kind, o->tma_box))
            dk.tm_base[0] = src;
        cudaError_t e = o->step(dk, src, states + k * lb, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The n reverse steps of one segment on the handle's stream, from the last
// level down, alternating between lam and lam_tmp so that lambda_{t0} lands
// in lam.
static cudaError_t adj_reverse_issue(lbm_sim *s, int64_t n, char *states, size_t lb, void *lam,
                                     void *lam_tmp, void *work) {
    const size_t sb = level_state_bytes(s->d, s->ops);
    void *in = lam, *out = lam_tmp;
    if (n % 2 == 1) {  // an odd count ends in lam only if it starts from lam_tmp
        cudaError_t e = cudaMemcpyAsync(lam_tmp, lam, sb, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return e;
        in = lam_tmp;
        out = lam;
    }
    const lbm::AdjHost h = adj_host(s->prm);
    for (int64_t k = n - 1; k >= 0; --k) {
        cudaError_t e = s->ops->adj_step(s->d, h, states + k * lb, in, out, work, s->stream);
        if (e != cudaSuccess) return e;
        void *t = in;
        in = out;
        out = t;
    }
    return cudaSuccess;
}

// The launch sequence of one segment: its recompute, then its reverse steps.
static cudaError_t adj_segment_issue(lbm_sim *s, int64_t n, char *states, size_t lb, void *lam,
                                     void *lam_tmp, void *work) {
    cudaError_t e = adj_recompute_issue(s, n, states, lb, s->stream);
    return e != cudaSuccess ? e : adj_reverse_issue(s, n, states, lb, lam, lam_tmp, work);
}

// The overlapped pair: the recompute of the next segment on the side stream
// (forked after everything issued so far on the handle's stream, so after
// the caller's copy of its checkpoint) and the reverse steps of this one on
// the handle's stream, joined at the end.
static cudaError_t adj_overlap_issue(lbm_sim *s, int64_t n, char *states, size_t lb, void *lam,
                                     void *lam_tmp, void *work, int64_t n_next, char *next_states) {
    cudaError_t e = cudaSuccess;
    if (n_next > 1) {
        if ((e = cudaEventRecord(s->adj_fork, s->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s->adj_side, s->adj_fork, 0)) != cudaSuccess) return e;
        if ((e = adj_recompute_issue(s, n_next, next_states, lb, s->adj_side)) != cudaSuccess) return e;
    }
    e = adj_reverse_issue(s, n, states, lb, lam, lam_tmp, work);
    if (n_next > 1) {
        // join even after a failed issue, so that no capture is left forked
        const cudaError_t e1 = cudaEventRecord(s->adj_join, s->adj_side);
        const cudaError_t e2 = cudaStreamWaitEvent(s->stream, s->adj_join, 0);
        if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    return e;
}

lbm_status lbm_adj_segment(lbm_sim *s, int64_t n, void *states, size_t level_stride, void *lam,
                           void *lam_tmp, void *work) {
    lbm::NvtxRange r_call("lbm_adj_segment");
    if (lbm_status st = adj_ready(s, work)) return st;
    if (!states || !lam || !lam_tmp) return s->fail(LBM_ERR_ARG, "null pointer");
    if (lam == lam_tmp) return s->fail(LBM_ERR_ARG, "lam and lam_tmp must differ");
    if (n < 1) return s->fail(LBM_ERR_ARG, "a segment needs at least one step");
    const size_t sb = level_state_bytes(s->d, s->ops);
    if (level_stride < sb || (level_stride & 255) || (reinterpret_cast<uintptr_t>(states) & 255))
        return s->fail(LBM_ERR_ARG, "level_stride must be >= lbm_state_bytes and states and "
                                    "level_stride 256-byte aligned");
    char *st_base = static_cast<char *>(states);
    if (!s->adj_graph) {
        LBM_CK(s, adj_segment_issue(s, n, st_base, level_stride, lam, lam_tmp, work));
        return LBM_OK;
    }
    const void *key[4] = {states, lam, lam_tmp, work};
    bool same = s->adj_exec && s->adj_n == n && s->adj_stride == level_stride;
    for (int i = 0; i < 4 && same; ++i) same = s->adj_key[i] == key[i];
    if (!same) {
        if (s->adj_exec) {
            cudaGraphExecDestroy(s->adj_exec);
            s->adj_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        LBM_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ei = adj_segment_issue(s, n, st_base, level_stride, lam, lam_tmp, work);
        const cudaError_t ec = cudaStreamEndCapture(s->stream, &g);
        if (ei != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return s->cuda(ei != cudaSuccess ? ei : ec, "capture of an adjoint segment");
        }
        const cudaError_t eg = cudaGraphInstantiate(&s->adj_exec, g, 0);
        cudaGraphDestroy(g);
        if (eg != cudaSuccess) {
            s->adj_exec = nullptr;
            return s->cuda(eg, "instantiation of an adjoint segment graph");
        }
        s->adj_n = n;
        s->adj_stride = level_stride;
        for (int i = 0; i < 4; ++i) s->adj_key[i] = key[i];
    }
    LBM_CK(s, cudaGraphLaunch(s->adj_exec, s->stream));
    return LBM_OK;
}

static lbm_status adj_states_ok(lbm_sim *s, const void *states, size_t level_stride) {
    const size_t sb = level_state_bytes(s->d, s->ops);
    if (!states) return s->fail(LBM_ERR_ARG, "null pointer");
    if (level_stride < sb || (level_stride & 255) || (reinterpret_cast<uintptr_t>(states) & 255))
        return s->fail(LBM_ERR_ARG, "level_stride must be >= lbm_state_bytes and states and "
                                    "level_stride 256-byte aligned");
    return LBM_OK;
}

lbm_status lbm_adj_recompute(lbm_sim *s, int64_t n, void *states, size_t level_stride) {
    lbm::NvtxRange r_call("lbm_adj_recompute");
    if (!s) return LBM_ERR_ARG;
    if (!s->ops->adj_step || s->d.lag) return s->fail(LBM_ERR_ARG, "no adjoint for this handle");
    if (n < 1) return s->fail(LBM_ERR_ARG, "a segment needs at least one step");
    if (lbm_status st = adj_states_ok(s, states, level_stride)) return st;
    LBM_CK(s, adj_recompute_issue(s, n, static_cast<char *>(states), level_stride, s->stream));
    return LBM_OK;
}

lbm_status lbm_adj_reverse_overlap(lbm_sim *s, int64_t n, void *states, size_t level_stride,
                                   void *lam, void *lam_tmp, void *work, int64_t n_next,
                                   void *next_states) {
    lbm::NvtxRange r_call("lbm_adj_reverse_overlap");
    if (lbm_status st = adj_ready(s, work)) return st;
    if (!lam || !lam_tmp) return s->fail(LBM_ERR_ARG, "null pointer");
    if (lam == lam_tmp) return s->fail(LBM_ERR_ARG, "lam and lam_tmp must differ");
    if (n < 1 || n_next < 0) return s->fail(LBM_ERR_ARG, "n >= 1 and n_next >= 0 required");
    if (lbm_status st = adj_states_ok(s, states, level_stride)) return st;
    if (n_next > 0) {
        if (lbm_status st = adj_states_ok(s, next_states, level_stride)) return st;
        if (next_states == states) return s->fail(LBM_ERR_ARG, "states and next_states must differ");
    }
    if (n_next > 1 && !s->adj_side) {
        LBM_CK(s, cudaStreamCreateWithFlags(&s->adj_side, cudaStreamNonBlocking));
        LBM_CK(s, cudaEventCreateWithFlags(&s->adj_fork, cudaEventDisableTiming));
        LBM_CK(s, cudaEventCreateWithFlags(&s->adj_join, cudaEventDisableTiming));
    }
    char *st_base = static_cast<char *>(states);
    char *nx_base = static_cast<char *>(next_states);
    if (!s->adj_graph) {
        LBM_CK(s, adj_overlap_issue(s, n, st_base, level_stride, lam, lam_tmp, work, n_next, nx_base));
        return LBM_OK;
    }
    const void *key[5] = {states, next_states, lam, lam_tmp, work};
    lbm_sim::OvGraph *hit = nullptr;
    for (auto &g : s->adj_ov) {
        bool same = g.exec && g.n == n && g.n_next == n_next && g.stride == level_stride;
        for (int i = 0; i < 5 && same; ++i) same = g.key[i] == key[i];
        if (same) hit = &g;
    }
    if (!hit) {
        hit = &s->adj_ov[s->adj_ov_next];
        s->adj_ov_next = 1 - s->adj_ov_next;
        if (hit->exec) {
            cudaGraphExecDestroy(hit->exec);
            hit->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        LBM_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ei =
            adj_overlap_issue(s, n, st_base, level_stride, lam, lam_tmp, work, n_next, nx_base);
        const cudaError_t ec = cudaStreamEndCapture(s->stream, &g);
        if (ei != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return s->cuda(ei != cudaSuccess ? ei : ec, "capture of an overlapped adjoint segment");
        }
        const cudaError_t eg = cudaGraphInstantiate(&hit->exec, g, 0);
        cudaGraphDestroy(g);
        if (eg != cudaSuccess) {
            hit->exec = nullptr;
            return s->cuda(eg, "instantiation of an overlapped adjoint segment graph");
        }
        hit->n = n;
        hit->n_next = n_next;
        hit->stride = level_stride;
        for (int i = 0; i < 5; ++i) hit->key[i] = key[i];
    }
    LBM_CK(s, cudaGraphLaunch(hit->exec, s->stream));
    return LBM_OK;
}

lbm_status lbm_adj_grads(lbm_sim *s, void *work, double *dM, double *dsigma) {
    if (lbm_status st = adj_ready(s, work)) return st;
    double h[2];
    const char *acc = static_cast<const char *>(work) + lbm::adj_acc_offset(s->d.NS, s->ops->field_size);
    LBM_CK(s, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    if (dM) *dM = h[0];
    if (dsigma) *dsigma = h[1];
    return LBM_OK;
}

}  // extern "C"
