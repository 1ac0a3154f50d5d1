// lbm_batch.cu — the batched form of the C ABI (include/lbm.h, lbm_batch_*).
//
// Many independent domains (each with its own size and parameters, one
// storage type for the whole batch) advance together: per time step one
// persistent launch of the batched strip kernel works through a list of
// (domain, strip, segment) items (the narrow-strip kernel when every strip
// has at most 64 active columns).  Optionally the launches are replayed
// from a CUDA graph.  Host-side bookkeeping only; every step of
// the method runs in the kernels of lbm_strip.cuh / lbm_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using lbm::BatchItem;
using lbm::Derived;
using lbm::Ops;
using lbm::derive;
using lbm::ops_for;

namespace {

constexpr int kMinSeg = 16;            // smallest segment height the item table is sized for
constexpr int kPartBlocks = 152 * 4;   // per-domain mass reduction grid

size_t r256(size_t b) { return (b + 255) & ~size_t(255); }

struct Plan {
    std::vector<Derived> d;
    std::vector<long long> lvl_off[2];  // byte offsets of each domain's two levels
    std::vector<long long> cell_off;    // first cell of each domain in concatenated fields
    long long cells = 0;
    size_t state = 0;
    // work buffer layout
    size_t doms_off = 0, items_off = 0, tickets_off = 0, fields_off = 0, field_slot = 0, part_off = 0,
           out_off = 0, work = 0;
    int max_items = 0;
};

std::string make_plan(const lbm_params *prms, int n, Plan &P, const Ops **ops_out) {
    if (!prms || n < 1) return "need at least one domain";
    const Ops *ops = ops_for(prms[0].dtype);
    if (!ops) return "unknown dtype";
    if (lbm::is_deviation_dtype(prms[0].dtype))
        return "the deviation storage (LBM_F16D, LBM_BF16D) runs single domains only";
    for (int i = 0; i < n; ++i) {
        size_t sb = 0, wb = 0;
        if (lbm_buffer_sizes(&prms[i], &sb, &wb) != LBM_OK)
            return "domain " + std::to_string(i) + ": " + lbm_create_error();
        if (prms[i].dtype != prms[0].dtype) return "all domains of a batch share one dtype";
        if (prms[i].gradp_lag) return "batched domains take the synchronous step (gradp_lag = 0)";
        Derived d = derive(&prms[i]);
        if (!ops->strip_ok(d))
            return "domain " + std::to_string(i) + ": batched domains need nx a multiple of 8";
        P.d.push_back(d);
    }
    size_t off = 0;
    P.lvl_off[0].resize(n);
    P.lvl_off[1].resize(n);
    P.cell_off.resize(n);
    long long items = 0;
    const int SW = ops->strip_width;
    for (int i = 0; i < n; ++i) {
        const size_t lv = r256(ops->level_bytes(P.d[i].NS));
        P.lvl_off[0][i] = (long long)off;
        P.lvl_off[1][i] = (long long)(off + lv);
        off += 2 * lv;
        P.cell_off[i] = P.cells;
        P.cells += P.d[i].N;
        items += (long long)((P.d[i].nx + SW - 1) / SW) * ((P.d[i].ny + kMinSeg - 1) / kMinSeg);
    }
    if (items > (1LL << 30)) return "too many work items";
    P.max_items = (int)items;
    P.state = off;
    size_t w = 0;
    P.doms_off = w;
    w += r256((size_t)n * ops->batch_dom_bytes);
    P.items_off = w;
    w += r256((size_t)P.max_items * sizeof(BatchItem));
    P.tickets_off = w;  // the work-claim counters of the two batch kernels
    w += 256;
    P.field_slot = r256((size_t)P.cells * ops->field_size);
    P.fields_off = w;
    w += 4 * P.field_slot;  // phi, ux, uy, p staging for host transfers
    P.part_off = w;
    w += r256((size_t)kPartBlocks * 2 * sizeof(double));
    P.out_off = w;
    w += r256((size_t)n * 2 * sizeof(double));
    P.work = w;
    *ops_out = ops;
    return "";
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_params> prm;
    Plan P;
    const Ops *ops = nullptr;
    cudaStream_t stream = nullptr;
    char *state = nullptr, *work = nullptr;
    int parity = 0;
    int64_t steps = 0;
    bool initialized = false;
    int seg_h = 64;
    int nitems = 0;    // items of more than narrow_width active columns
    int nitems_n = 0;  // items of at most narrow_width active columns
    bool items_ready = false;
    bool use_graph = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two steps starting at parity 0 / 1
    std::string err;

    lbm_status fail(lbm_status s, const std::string &m) {
        err = m;
        return s;
    }
    lbm_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return LBM_OK;
        err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
        return LBM_ERR_CUDA;
    }
    void drop_graphs() {
        for (auto &g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    char *level(int dom, int par) { return state + P.lvl_off[par][dom]; }
    BatchItem *items() { return reinterpret_cast<BatchItem *>(work + P.items_off); }
    unsigned long long *tickets() { return reinterpret_cast<unsigned long long *>(work + P.tickets_off); }
    char *slot(int i) { return work + P.fields_off + (size_t)i * P.field_slot; }
};

#define LBMB_CK(b, call)                                   \
    do {                                                   \
        lbm_status st__ = (b)->cuda((call), #call);        \
        if (st__ != LBM_OK) return st__;                   \
    } while (0)

namespace {

// The work list for segment height seg_h.  A strip of at most narrow_width
// active columns counts as narrow when the form has a narrow kernel (used
// only when every strip is narrow).  The persistent grid's CTAs claim items
// in list order.  Each domain's items stay together, domains in order of
// decreasing longest item, so that the strips and segments of one domain
// run at the same time and share in L2 the halo columns and warm-up rows
// they both read, and the sectors both write at a strip edge: at segment
// height 96 the 1024-domain workload moved 1.13x its algorithmic DRAM bytes
// per step, against 1.21x with all items sorted longest first (wide, then
// narrow).
lbm_status build_items(lbm_batch *b) {
    const int SW = b->ops->strip_width;
    const int NW = b->ops->batch_step_narrow ? b->ops->narrow_width : 0;
    const size_t nd = b->P.d.size();
    std::vector<std::vector<BatchItem>> per(nd);
    std::vector<long long> dcost(nd, 0);
    int nwide = 0, nnarrow = 0;
    for (size_t i = 0; i < nd; ++i) {
        const Derived &d = b->P.d[i];
        const int nseg = (d.ny + b->seg_h - 1) / b->seg_h;
        const int h = (d.ny + nseg - 1) / nseg;  // balanced segment height
        for (int x0 = 0; x0 < d.nx; x0 += SW) {
            const int w = std::min(SW, d.nx - x0);
            for (int ys = 0; ys < d.ny; ys += h) {
                const int ye = std::min(ys + h, d.ny);
                const long long c = (long long)w * (ye - ys + 6);
                per[i].push_back(BatchItem{(int)i, x0, ys, ye});
                dcost[i] = std::max(dcost[i], c);
                ++(w <= NW ? nnarrow : nwide);
            }
        }
    }
    if (nwide + nnarrow > b->P.max_items)
        return b->fail(LBM_ERR_ARG, "segment height too small");
    std::vector<BatchItem> sorted;
    sorted.reserve((size_t)(nwide + nnarrow));
    std::vector<int> order(nd);
    for (size_t i = 0; i < nd; ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return dcost[a] > dcost[c]; });
    for (int o : order) sorted.insert(sorted.end(), per[o].begin(), per[o].end());
    LBMB_CK(b, cudaMemcpyAsync(b->items(), sorted.data(), sorted.size() * sizeof(BatchItem),
                               cudaMemcpyHostToDevice, b->stream));
    // new item counts change the tickets per step: restart both counters
    LBMB_CK(b, cudaMemsetAsync(b->tickets(), 0, 2 * sizeof(unsigned long long), b->stream));
    LBMB_CK(b, cudaStreamSynchronize(b->stream));
    b->nitems = nwide;
    b->nitems_n = nnarrow;
    b->items_ready = true;
    b->drop_graphs();
    return LBM_OK;
}

// One step, one launch.  A batch whose strips are all narrow (at most
// narrow_width active columns) runs the narrow kernel over them; any other
// batch runs the strip_width kernel over every item, wide ones first.  On
// the 1024-domain workload (FP32) this single launch measured 32.0k MLUPS;
// two launches per step, the narrow items on the narrow kernel after the
// wide ones, 31.3k; one launch that ran the narrow items two per CTA, a
// half CTA each, spilled registers and measured 27.3k.
lbm_status launch_step(lbm_batch *b, int parity) {
    const void *doms = b->work + b->P.doms_off;
    lbm::NvtxRange r_launch("batch step");
    const int n = b->nitems + b->nitems_n;
    if (n == 0) return LBM_OK;
    int slots = 0;
    if (b->nitems == 0 && b->ops->batch_step_narrow) {
        LBMB_CK(b, b->ops->batch_slots_narrow(&slots));
        LBMB_CK(b, b->ops->batch_step_narrow(b->state, doms, b->items(), n, b->tickets() + 1, parity,
                                             std::min(slots, n), b->stream));
    } else {
        LBMB_CK(b, b->ops->batch_slots(&slots));
        LBMB_CK(b, b->ops->batch_step(b->state, doms, b->items(), n, b->tickets(), parity,
                                      std::min(slots, n), b->stream));
    }
    return LBM_OK;
}

lbm_status capture_pair(lbm_batch *b, int first) {
    cudaGraph_t g = nullptr;
    LBMB_CK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = launch_step(b, first);
    if (st == LBM_OK) st = launch_step(b, 1 - first);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    LBMB_CK(b, e);
    e = cudaGraphInstantiate(&b->graph[first], g, 0);
    cudaGraphDestroy(g);
    LBMB_CK(b, e);
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_buffer_sizes(const lbm_params *prms, int n, size_t *state_bytes,
                                  size_t *work_bytes) {
    Plan P;
    const Ops *ops = nullptr;
    std::string m = make_plan(prms, n, P, &ops);
    if (!m.empty()) {
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    if (state_bytes) *state_bytes = P.state;
    if (work_bytes) *work_bytes = P.work;
    return LBM_OK;
}

lbm_status lbm_batch_create(const lbm_params *prms, int n, void *stream, lbm_batch **out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_NOMEM;
    std::string m = make_plan(prms, n, b->P, &b->ops);
    if (!m.empty()) {
        delete b;
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    b->prm.assign(prms, prms + n);
    b->stream = static_cast<cudaStream_t>(stream);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_bind_buffers(lbm_batch *b, void *state, size_t state_bytes, void *work,
                                  size_t work_bytes) {
    if (!b) return LBM_ERR_ARG;
    if (!state || !work) return b->fail(LBM_ERR_ARG, "null buffer");
    if ((reinterpret_cast<uintptr_t>(state) & 255) || (reinterpret_cast<uintptr_t>(work) & 255))
        return b->fail(LBM_ERR_ARG, "buffers must be 256-byte aligned");
    if (state_bytes < b->P.state || work_bytes < b->P.work)
        return b->fail(LBM_ERR_NOMEM, "bound buffer smaller than lbm_batch_buffer_sizes");
    b->state = static_cast<char *>(state);
    b->work = static_cast<char *>(work);
    b->drop_graphs();
    int slots = 0;  // sets the kernels' shared-memory attribute outside any capture
    LBMB_CK(b, b->ops->batch_slots(&slots));
    if (b->ops->batch_step_narrow) LBMB_CK(b, b->ops->batch_slots_narrow(&slots));
    // domain table
    const size_t db = b->ops->batch_dom_bytes;
    std::vector<char> host(b->P.d.size() * db);
    for (size_t i = 0; i < b->P.d.size(); ++i)
        b->ops->batch_fill_dom(host.data() + i * db, b->P.d[i], b->P.lvl_off[0][i],
                               b->P.lvl_off[1][i]);
    LBMB_CK(b, cudaMemcpyAsync(b->work + b->P.doms_off, host.data(), host.size(),
                               cudaMemcpyHostToDevice, b->stream));
    LBMB_CK(b, cudaStreamSynchronize(b->stream));
    b->initialized = false;
    return build_items(b);
}

lbm_status lbm_batch_init_phi(lbm_batch *b, const void *phi, int on_host) {
    if (!b) return LBM_ERR_ARG;
    if (!b->state) return b->fail(LBM_ERR_STATE, "buffers not bound");
    if (!phi) return b->fail(LBM_ERR_ARG, "phi is null");
    const size_t fs = b->ops->field_size;
    const char *src = static_cast<const char *>(phi);
    if (on_host) {
        LBMB_CK(b, cudaMemcpyAsync(b->slot(0), phi, (size_t)b->P.cells * fs,
                                   cudaMemcpyHostToDevice, b->stream));
        src = b->slot(0);
    }
    for (size_t i = 0; i < b->P.d.size(); ++i)
        LBMB_CK(b, b->ops->init(b->P.d[i], src + (size_t)b->P.cell_off[i] * fs, nullptr, nullptr,
                                b->level((int)i, 0), b->stream));
    if (on_host) LBMB_CK(b, cudaStreamSynchronize(b->stream));
    b->parity = 0;
    b->steps = 0;
    b->initialized = true;
    return LBM_OK;
}

lbm_status lbm_batch_set_graph(lbm_batch *b, int use_graph) {
    if (!b) return LBM_ERR_ARG;
    if (use_graph && b->stream == nullptr)
        return b->fail(LBM_ERR_ARG, "graph replay needs a non-default stream");
    b->use_graph = use_graph != 0;
    b->drop_graphs();
    return LBM_OK;
}

lbm_status lbm_batch_set_segment(lbm_batch *b, int seg_h) {
    if (!b) return LBM_ERR_ARG;
    if (seg_h < kMinSeg) return b->fail(LBM_ERR_ARG, "segment height below 16");
    if (!b->state) return b->fail(LBM_ERR_STATE, "buffers not bound");
    b->seg_h = seg_h;
    return build_items(b);
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t n) {
    lbm::NvtxRange r_call("lbm_batch_step");
    if (!b) return LBM_ERR_ARG;
    if (!b->initialized) return b->fail(LBM_ERR_STATE, "lbm_batch_step before lbm_batch_init_phi");
    if (n < 0) return b->fail(LBM_ERR_ARG, "negative step count");
    while (n > 0) {
        if (b->use_graph && n >= 2) {
            if (!b->graph[b->parity])
                if (lbm_status st = capture_pair(b, b->parity)) return st;
            LBMB_CK(b, cudaGraphLaunch(b->graph[b->parity], b->stream));
            b->steps += 2;  // parity unchanged after two steps
            n -= 2;
        } else {
            if (lbm_status st = launch_step(b, b->parity)) return st;
            b->parity = 1 - b->parity;
            b->steps += 1;
            n -= 1;
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *seg_h_out, double *ms_out) {
    if (!b) return LBM_ERR_ARG;
    if (!b->initialized) return b->fail(LBM_ERR_STATE, "autotune needs an initialised state");
    if (steps < 1) steps = 1;
    static const int cand[] = {16, 24, 32, 48, 64, 96, 128, 192, 256};
    cudaEvent_t e0, e1;
    LBMB_CK(b, cudaEventCreate(&e0));
    LBMB_CK(b, cudaEventCreate(&e1));
    const bool graph = b->use_graph;
    b->use_graph = false;
    int best = b->seg_h;
    float best_ms = 1e30f;
    lbm_status st = LBM_OK;
    for (int c : cand) {
        b->seg_h = c;
        if ((st = build_items(b)) != LBM_OK) break;
        if ((st = lbm_batch_step(b, 1)) != LBM_OK) break;  // warm-up
        cudaEventRecord(e0, b->stream);
        if ((st = lbm_batch_step(b, steps)) != LBM_OK) break;
        cudaEventRecord(e1, b->stream);
        if ((st = b->cuda(cudaEventSynchronize(e1), "cudaEventSynchronize")) != LBM_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= steps;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->use_graph = graph;
    if (st != LBM_OK) return st;
    b->seg_h = best;
    if ((st = build_items(b)) != LBM_OK) return st;
    if (seg_h_out) *seg_h_out = best;
    if (ms_out) *ms_out = best_ms;
    return LBM_OK;
}

lbm_status lbm_batch_fields(lbm_batch *b, void *phi, void *ux, void *uy, void *p, int on_host) {
    if (!b) return LBM_ERR_ARG;
    if (!b->initialized) return b->fail(LBM_ERR_STATE, "lbm_batch_fields before init");
    const size_t fs = b->ops->field_size;
    void *user[4] = {phi, ux, uy, p};
    char *dev[4];
    for (int k = 0; k < 4; ++k)
        dev[k] = on_host ? (user[k] ? b->slot(k) : nullptr) : static_cast<char *>(user[k]);
    for (size_t i = 0; i < b->P.d.size(); ++i) {
        const size_t o = (size_t)b->P.cell_off[i] * fs;
        auto at = [&](int k) -> void * { return dev[k] ? dev[k] + o : nullptr; };
        LBMB_CK(b, b->ops->fields(b->P.d[i], b->level((int)i, b->parity), at(0), nullptr, at(3),
                                  at(1), at(2), nullptr, nullptr, b->stream));
    }
    if (on_host) {
        for (int k = 0; k < 4; ++k)
            if (user[k])
                LBMB_CK(b, cudaMemcpyAsync(user[k], dev[k], (size_t)b->P.cells * fs,
                                           cudaMemcpyDeviceToHost, b->stream));
        LBMB_CK(b, cudaStreamSynchronize(b->stream));
    }
    return LBM_OK;
}

lbm_status lbm_batch_mass(lbm_batch *b, double *mass, double *phi_total) {
    if (!b) return LBM_ERR_ARG;
    if (!b->initialized) return b->fail(LBM_ERR_STATE, "lbm_batch_mass before init");
    const int n = (int)b->P.d.size();
    double *part = reinterpret_cast<double *>(b->work + b->P.part_off);
    double *out = reinterpret_cast<double *>(b->work + b->P.out_off);
    for (int i = 0; i < n; ++i) {
        const long long nb = (b->P.d[i].N + 255) / 256;
        const int nblocks = (int)std::min<long long>(nb, kPartBlocks);
        LBMB_CK(b, b->ops->mass(b->P.d[i], b->level(i, b->parity), part, nblocks, out + 2 * i,
                                b->stream));
    }
    std::vector<double> h((size_t)2 * n);
    LBMB_CK(b, cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               b->stream));
    LBMB_CK(b, cudaStreamSynchronize(b->stream));
    bool finite = true;
    for (int i = 0; i < n; ++i) {
        if (mass) mass[i] = h[2 * i];
        if (phi_total) phi_total[i] = h[2 * i + 1];
        finite = finite && std::isfinite(h[2 * i]) && std::isfinite(h[2 * i + 1]);
    }
    if (!finite) return b->fail(LBM_ERR_NONFINITE, "non-finite mass or phi total");
    return LBM_OK;
}

int64_t lbm_batch_cells(const lbm_batch *b) { return b ? b->P.cells : 0; }

int64_t lbm_batch_step_count(const lbm_batch *b) { return b ? b->steps : 0; }

int lbm_batch_segment(const lbm_batch *b) { return b ? b->seg_h : 0; }

lbm_status lbm_batch_work_items(const lbm_batch *b, int *wide, int *narrow) {
    if (!b) return LBM_ERR_ARG;
    if (!b->items_ready) return LBM_ERR_STATE;
    if (wide) *wide = b->nitems;
    if (narrow) *narrow = b->nitems_n;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : "null handle"; }

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    b->drop_graphs();
    delete b;
}

}  // extern "C"
