// lbm_slabs.cu — one domain decomposed into y-slabs (include/lbm.h,
// lbm_slabs_*): the domain decomposition the step shards by, with every
// slab on this device and device-to-device ghost-row exchange.
//
// Slab i owns global rows a_i .. b_i-1 and holds them with 3 ghost rows on
// each side (the step's reach in y: grad p <- p <- lap mu <- lap phi <- g).
// One time step is
//   1. the strip kernel on every slab, rows a_i .. b_i-1 only, reading the
//      ghost rows and pushing across its edges into them (KP::slab);
//   2. the crossing copy: populations pushed across an edge (slots with
//      c_y = +1: 2, 5, 6 of f and g upward; c_y = -1: 4, 7, 8 downward)
//      move from the ghost row they landed in to the slab that owns it;
//   3. the halo copy: every slab's 3 ghost rows on each side receive all 18
//      slots of the neighbour's 3 edge rows.
// Steps 2 and 3 are one launch each of k_copy_spans over precomputed
// (source, destination, bytes) tables, one table per ping-pong parity.
// Each cell goes through the same kernel body and arithmetic as in the
// whole-domain step, so results are bit-identical to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using lbm::Derived;
using lbm::Ops;

namespace {

constexpr int kGhost = 3;  // ghost rows per side
// copy spans per slab edge and parity: 12 crossing (slots 2, 5, 6 up and
// 4, 7, 8 down, of f and of g), then 36 halo (18 slots, both directions)
constexpr int kCrossPerEdge = 12, kHaloPerEdge = 36;
constexpr int kSpansPerEdge = kCrossPerEdge + kHaloPerEdge;

size_t r256(size_t b) { return (b + 255) & ~size_t(255); }

struct Span {
    const char *src;
    char *dst;
    long long bytes;  // multiple of 16; both addresses 16-byte aligned
};

// Copies every span of the table; blockIdx.y walks the spans.
__global__ void k_copy_spans(const Span *__restrict__ spans, int n) {
    for (int s = blockIdx.y; s < n; s += gridDim.y) {
        const Span c = spans[s];
        const int4 *src = reinterpret_cast<const int4 *>(c.src);
        int4 *dst = reinterpret_cast<int4 *>(c.dst);
        const long long n16 = c.bytes >> 4;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
             i += (long long)gridDim.x * blockDim.x)
            dst[i] = src[i];
    }
}

struct Plan {
    Derived d;                     // the whole domain
    std::vector<int> a, b;         // rows owned by each slab
    std::vector<Derived> ds;       // per slab: NS, y0, rows, ya, yb
    std::vector<size_t> lvl_off;   // byte offset of slab i's level 0 (level 1 follows)
    std::vector<size_t> lvl_bytes;
    size_t state = 0;
    int boundaries = 0;            // slab edges that exchange (periodic: n, walls: n - 1)
    size_t work = 0;
};

std::string make_plan(const lbm_params *p, int n, const int *starts, Plan &P, const Ops **ops_out) {
    std::string m = lbm::check_params(p);
    if (!m.empty()) return m;
    if (p->gradp_lag) return "slabs take the synchronous step (gradp_lag = 0)";
    if (lbm::is_deviation_dtype(p->dtype))
        return "the deviation storage (LBM_F16D, LBM_BF16D) runs single domains only";
    const Ops *ops = lbm::ops_for(p->dtype);
    P.d = lbm::derive(p);
    if (n < 1) return "need at least one slab";
    if (n > P.d.ny / kGhost) return "too many slabs for ny (each needs >= 3 rows)";
    P.a.resize(n);
    P.b.resize(n);
    for (int i = 0; i < n; ++i) {
        P.a[i] = starts ? starts[i] : (int)((long long)P.d.ny * i / n);
        P.b[i] = i + 1 < n ? (starts ? starts[i + 1] : (int)((long long)P.d.ny * (i + 1) / n))
                           : P.d.ny;
    }
    if (P.a[0] != 0) return "row_starts[0] must be 0";
    for (int i = 0; i < n; ++i)
        if (P.b[i] - P.a[i] < kGhost) return "every slab needs >= 3 rows (increasing row_starts)";
    P.ds.resize(n);
    P.lvl_off.resize(n);
    P.lvl_bytes.resize(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        Derived s = P.d;
        s.slab = 1;
        s.y0 = P.a[i] - kGhost;
        s.rows = P.b[i] - P.a[i] + 2 * kGhost;
        s.ya = P.a[i];
        s.yb = P.b[i];
        s.N = (long long)s.rows * s.nx;
        s.NS = (s.N + 127) / 128 * 128;
        s.share = n;  // the slabs of a step run at the same time
        if (!ops->strip_ok(s)) return "slabs need nx a multiple of 8";
        P.ds[i] = s;
        P.lvl_bytes[i] = r256(ops->level_bytes(s.NS));
        P.lvl_off[i] = off;
        off += 2 * P.lvl_bytes[i];
    }
    P.state = off;
    P.boundaries = P.d.wall ? n - 1 : n;
    P.work = 2 * r256((size_t)P.boundaries * kSpansPerEdge * sizeof(Span)) + 256;
    *ops_out = ops;
    return "";
}

const int kUp[3] = {2, 5, 6};    // c_y = +1
const int kDown[3] = {4, 7, 8};  // c_y = -1

}  // namespace

struct lbm_slabs {
    Plan P;
    const Ops *ops = nullptr;
    cudaStream_t stream = nullptr;
    char *state = nullptr;
    Span *tables = nullptr;  // device: parity 0 then parity 1, each cross then halo
    int n_cross = 0, n_halo = 0;
    size_t table_stride = 0;  // spans per parity
    int cur = 0;
    int64_t steps = 0;
    bool initialized = false;
    // slabs 1..n-1 step on side streams forked from and joined to `stream`
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    std::string err;
    ~lbm_slabs() {
        for (cudaStream_t t : side) cudaStreamDestroy(t);
        for (cudaEvent_t e : done) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
    lbm_status fail(lbm_status st, const std::string &m) {
        err = m;
        return st;
    }
    lbm_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return LBM_OK;
        return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    int n() const { return (int)P.a.size(); }
    char *level(int i, int lv) const { return state + P.lvl_off[i] + (size_t)lv * P.lvl_bytes[i]; }
    // address of global row y (a row the slab holds) of slot q in level lv of slab i
    char *row_ptr(int i, int lv, int q, int y) const {
        size_t off = 0, elem = 0;
        ops->slot_span(P.ds[i].NS, q, &off, &elem);
        return level(i, lv) + off + (size_t)(y - P.ds[i].y0) * P.d.nx * elem;
    }
    size_t row_bytes(int q) const {
        size_t off = 0, elem = 0;
        ops->slot_span(P.d.NS, q, &off, &elem);
        return (size_t)P.d.nx * elem;
    }
};

static lbm_status bind_tables(lbm_slabs *s, char *state, void *work);

extern "C" {

lbm_status lbm_slabs_buffer_sizes(const lbm_params *prm, int n_slabs, const int *row_starts,
                                  size_t *state_bytes, size_t *work_bytes) {
    Plan P;
    const Ops *ops = nullptr;
    std::string m = make_plan(prm, n_slabs, row_starts, P, &ops);
    if (!m.empty()) {
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    if (state_bytes) *state_bytes = P.state;
    if (work_bytes) *work_bytes = P.work;
    return LBM_OK;
}

lbm_status lbm_slabs_create(const lbm_params *prm, int n_slabs, const int *row_starts,
                            void *stream, lbm_slabs **out) {
    if (!out) {
        lbm_internal_set_error("null output handle");
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    lbm_slabs *s = new lbm_slabs();
    std::string m = make_plan(prm, n_slabs, row_starts, s->P, &s->ops);
    if (!m.empty()) {
        delete s;
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    s->stream = static_cast<cudaStream_t>(stream);
    *out = s;
    return LBM_OK;
}

lbm_status lbm_slabs_bind_buffers(lbm_slabs *s, void *state, size_t state_bytes, void *work,
                                  size_t work_bytes) {
    if (!s) return LBM_ERR_ARG;
    if (!state || !work) return s->fail(LBM_ERR_ARG, "null buffer");
    if (state_bytes < s->P.state || work_bytes < s->P.work)
        return s->fail(LBM_ERR_NOMEM, "bound buffer smaller than lbm_slabs_buffer_sizes");
    if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(work)) & 255)
        return s->fail(LBM_ERR_ARG, "buffers must be 256-byte aligned");
    const int n = s->n();
    // Side streams and events first, into locals: they join the handle only
    // when all n - 1 exist, so a failed bind leaves it as it was.
    if (!s->fork && n > 1) {
        cudaEvent_t fork = nullptr;
        std::vector<cudaStream_t> side;
        std::vector<cudaEvent_t> done;
        cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        for (int i = 1; i < n && e == cudaSuccess; ++i) {
            cudaStream_t t = nullptr;
            e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
            if (e != cudaSuccess) break;
            side.push_back(t);
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            done.push_back(ev);
        }
        if (e != cudaSuccess) {
            for (cudaStream_t t : side) cudaStreamDestroy(t);
            for (cudaEvent_t ev : done) cudaEventDestroy(ev);
            if (fork) cudaEventDestroy(fork);
            return s->cuda(e, "side streams of the slab steps");
        }
        s->fork = fork;
        s->side = std::move(side);
        s->done = std::move(done);
    }
    // The handle counts as bound (s->state set) only once the tables are
    // uploaded; scatter and step refuse it until then.
    s->state = nullptr;
    char *const st_base = static_cast<char *>(state);
    const lbm_status bound = bind_tables(s, st_base, work);
    s->state = bound == LBM_OK ? st_base : nullptr;
    // tensor maps of every slab's two levels (FP32): the slab steps take
    // their interior strips' rows as tensor tiles; a level without a map
    // is stepped with chunk copies
    for (int i = 0; i < n && bound == LBM_OK; ++i) {
        Derived &d = s->P.ds[i];
        for (int lv = 0; lv < 2; ++lv) {
            d.tm_base[lv] = nullptr;
            if (s->ops->tma_kind > 0 &&
                lbm::encode_level_maps(d.tm[lv], s->level(i, lv), d, s->ops->tma_kind, s->ops->tma_box))
                d.tm_base[lv] = s->level(i, lv);
        }
    }
    return bound;
}

}  // extern "C"

// Builds and uploads the span tables of both parities, and clears the
// state buffer; row addresses are taken relative to `state`.
static lbm_status bind_tables(lbm_slabs *s, char *state, void *work) {
    s->state = state;  // row_ptr addresses rows through it
    s->tables = reinterpret_cast<Span *>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
    const int n = s->n();
    // Span tables of both parities (the level written by the step).
    std::vector<Span> host;
    s->table_stride = (size_t)s->P.boundaries * kSpansPerEdge;
    host.resize(2 * s->table_stride);
    for (int lv = 0; lv < 2; ++lv) {
        Span *cross = host.data() + lv * s->table_stride;
        Span *halo = cross + kCrossPerEdge * s->P.boundaries;
        int nc = 0, nh = 0;
        for (int lo = 0; lo < s->P.boundaries; ++lo) {
            const int up = (lo + 1) % n;          // slab above the edge
            const int e = s->P.b[lo];   // first row above the edge, as slab lo numbers it
            const int eu = s->P.a[up];  // the same row as slab up numbers it (0 across the wrap)
            for (int k = 0; k < 3; ++k)
                for (int h = 0; h < 2; ++h) {  // f slot, g slot
                    const int q = kUp[k] + 9 * h;
                    cross[nc++] = {s->row_ptr(lo, lv, q, e), s->row_ptr(up, lv, q, eu),
                                   (long long)s->row_bytes(q)};
                    const int qd = kDown[k] + 9 * h;
                    cross[nc++] = {s->row_ptr(up, lv, qd, eu - 1), s->row_ptr(lo, lv, qd, e - 1),
                                   (long long)s->row_bytes(qd)};
                }
            for (int q = 0; q < 18; ++q) {
                const long long rb = 3 * (long long)s->row_bytes(q);
                halo[nh++] = {s->row_ptr(lo, lv, q, e - kGhost), s->row_ptr(up, lv, q, eu - kGhost), rb};
                halo[nh++] = {s->row_ptr(up, lv, q, eu), s->row_ptr(lo, lv, q, e), rb};
            }
        }
        s->n_cross = nc;
        s->n_halo = nh;
    }
    for (const Span &c : host)
        if (c.bytes && (((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst)) & 15) ||
                        (c.bytes & 15)))
            return s->fail(LBM_ERR_ARG, "slab rows are not 16-byte aligned");
    if (lbm_status st = s->cuda(cudaMemcpyAsync(s->tables, host.data(), host.size() * sizeof(Span),
                                                cudaMemcpyHostToDevice, s->stream),
                                "upload of the span tables"))
        return st;
    // ghost rows past a wall are never read; clear everything once anyway
    if (lbm_status st = s->cuda(cudaMemsetAsync(s->state, 0, s->P.state, s->stream), "memset"))
        return st;
    return s->cuda(cudaStreamSynchronize(s->stream), "bind");
}

extern "C" {

lbm_status lbm_slabs_scatter(lbm_slabs *s, const void *level, int64_t step) {
    if (!s) return LBM_ERR_ARG;
    if (!s->state) return s->fail(LBM_ERR_STATE, "lbm_slabs_scatter before lbm_slabs_bind_buffers");
    if (!level) return s->fail(LBM_ERR_ARG, "null level");
    const char *src = static_cast<const char *>(level);
    const int ny = s->P.d.ny, nx = s->P.d.nx;
    for (int i = 0; i < s->n(); ++i)
        for (int q = 0; q < 18; ++q) {
            size_t off = 0, elem = 0;
            s->ops->slot_span(s->P.d.NS, q, &off, &elem);
            // rows a-3 .. b+2, as runs of consecutive rows of the whole domain
            int y = s->P.a[i] - kGhost;
            const int y1 = s->P.b[i] + kGhost;
            while (y < y1) {
                int g = y, len = y1 - y;
                if (s->P.d.wall) {
                    if (y < 0) {  // past a wall: never read
                        y = 0;
                        continue;
                    }
                    if (y >= ny) break;
                    if (y + len > ny) len = ny - y;
                } else {
                    g = ((y % ny) + ny) % ny;
                    if (g + len > ny) len = ny - g;
                }
                cudaError_t e = cudaMemcpyAsync(s->row_ptr(i, 0, q, y),
                                                src + off + (size_t)g * nx * elem,
                                                (size_t)len * nx * elem, cudaMemcpyDeviceToDevice,
                                                s->stream);
                if (lbm_status st = s->cuda(e, "scatter")) return st;
                y += len;
            }
        }
    s->cur = 0;
    s->steps = step;
    s->initialized = true;
    return LBM_OK;
}

lbm_status lbm_slabs_gather(lbm_slabs *s, void *level, int64_t *step) {
    if (!s) return LBM_ERR_ARG;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_slabs_gather before lbm_slabs_scatter");
    if (!level) return s->fail(LBM_ERR_ARG, "null level");
    char *dst = static_cast<char *>(level);
    const int nx = s->P.d.nx;
    for (int i = 0; i < s->n(); ++i)
        for (int q = 0; q < 18; ++q) {
            size_t off = 0, elem = 0;
            s->ops->slot_span(s->P.d.NS, q, &off, &elem);
            const int a = s->P.a[i], b = s->P.b[i];
            cudaError_t e = cudaMemcpyAsync(dst + off + (size_t)a * nx * elem,
                                            s->row_ptr(i, s->cur, q, a), (size_t)(b - a) * nx * elem,
                                            cudaMemcpyDeviceToDevice, s->stream);
            if (lbm_status st = s->cuda(e, "gather")) return st;
        }
    if (step) *step = s->steps;
    return LBM_OK;
}

lbm_status lbm_slabs_step(lbm_slabs *s, int64_t n) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm_slabs_step");
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm_slabs_step before lbm_slabs_scatter");
    if (n < 0) return s->fail(LBM_ERR_ARG, "negative step count");
    for (int64_t t = 0; t < n; ++t) {
        const int nxt = 1 - s->cur;
        // the slab steps are independent: slab i > 0 runs on side stream i-1,
        // each launch sized for 1/n of the GPU (Derived::share), and the
        // exchange waits for all of them
        const bool par = !s->side.empty();
        if (par) {
            if (lbm_status st = s->cuda(cudaEventRecord(s->fork, s->stream), "fork")) return st;
            for (cudaStream_t t : s->side)
                if (lbm_status st = s->cuda(cudaStreamWaitEvent(t, s->fork, 0), "fork")) return st;
        }
        lbm::NvtxRange r_launch(s->ops->step_range);
        for (int i = 0; i < s->n(); ++i)
            if (lbm_status st = s->cuda(s->ops->step(s->P.ds[i], s->level(i, s->cur), s->level(i, nxt),
                                                     i == 0 || !par ? s->stream : s->side[i - 1]),
                                        "slab step"))
                return st;
        if (par)
            for (size_t j = 0; j < s->side.size(); ++j) {
                if (lbm_status st = s->cuda(cudaEventRecord(s->done[j], s->side[j]), "join")) return st;
                if (lbm_status st = s->cuda(cudaStreamWaitEvent(s->stream, s->done[j], 0), "join")) return st;
            }
        if (s->P.boundaries > 0) {
            const Span *tab = s->tables + nxt * s->table_stride;
            // enough CTAs in x to cover the largest span (3 FP64 rows) in one pass
            const int gx = (int)((3 * (long long)s->P.d.nx * 8 / 16 + 255) / 256);
            const unsigned gc = (unsigned)std::min(s->n_cross, 65535);
            const unsigned gh = (unsigned)std::min(s->n_halo, 65535);
            k_copy_spans<<<dim3(gx, gc), 256, 0, s->stream>>>(tab, s->n_cross);
            if (lbm_status st = s->cuda(cudaGetLastError(), "crossing copy")) return st;
            k_copy_spans<<<dim3(gx, gh), 256, 0, s->stream>>>(tab + s->n_cross, s->n_halo);
            if (lbm_status st = s->cuda(cudaGetLastError(), "halo copy")) return st;
        }
        s->cur = nxt;
        ++s->steps;
    }
    return LBM_OK;
}

lbm_status lbm_slabs_rows(const lbm_slabs *s, int i, int *a, int *b) {
    if (!s || i < 0 || i >= s->n()) return LBM_ERR_ARG;
    if (a) *a = s->P.a[i];
    if (b) *b = s->P.b[i];
    return LBM_OK;
}

int64_t lbm_slabs_step_count(const lbm_slabs *s) { return s ? s->steps : 0; }

const char *lbm_slabs_last_error(const lbm_slabs *s) { return s ? s->err.c_str() : "null handle"; }

void lbm_slabs_destroy(lbm_slabs *s) { delete s; }

}  // extern "C"
