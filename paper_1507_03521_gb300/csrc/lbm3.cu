// lbm3.cu — the C ABI of the three-dimensional (D3Q19) step, lbm3_* in
// include/lbm.h.  Host-side bookkeeping only: validation, the buffer
// layout and the launch sequence; every pass runs in lbm3_kernels.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "lbm.h"
#include "lbm3_kernels.cuh"
#include "lbm_internal.h"

using lbm3::K3;

namespace {

constexpr int kThreads = 256;
constexpr int kParts = 152 * 4;  // reduction grid

size_t r256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout3 {
    long long N, NS;
    size_t elem, level, field, part_off, out_off, work;
};

Layout3 layout3(long long N, size_t elem) {
    Layout3 L;
    L.N = N;
    L.NS = (N + 127) / 128 * 128;
    L.elem = elem;
    L.level = r256((size_t)38 * L.NS * elem);
    L.field = r256((size_t)L.NS * elem);
    L.part_off = 3 * L.field;  // phi, mu, p
    L.out_off = L.part_off + r256((size_t)kParts * 5 * sizeof(double));
    L.work = L.out_off + 256;
    return L;
}

std::string check3(const lbm_params *p, int nz) {
    std::string m = lbm::check_params(p);
    if (!m.empty()) return m;
    if (nz < 3) return "nz must be >= 3";
    if (p->bc_y != LBM_PERIODIC) return "the 3-D step is periodic in every direction";
    if (p->dtype != LBM_F32 && p->dtype != LBM_F64) return "the 3-D step supports LBM_F32 and LBM_F64";
    if (p->gradp_lag) return "the 3-D step is the synchronous scheme (gradp_lag = 0)";
    if ((long long)p->nx * p->ny * nz >= (1LL << 31)) return "grid too large for the 3-D step";
    if (p->ny > 65535 || nz > 65535) return "ny and nz must be <= 65535 for the 3-D step";
    return "";
}

template <class T>
K3<T> make_k3(const lbm::Derived &d, int nz, const Layout3 &L) {
    K3<T> k;
    k.nx = d.nx;
    k.ny = d.ny;
    k.nz = nz;
    k.N = L.N;
    k.NS = L.NS;
    k.phiA = T(d.phiA);
    k.phiB = T(d.phiB);
    k.phibar = T(d.phibar);
    k.rhoB = T(d.rhoB);
    k.drho = T(d.drho);
    k.kappa = T(d.kappa);
    k.beta4 = T(4.0 * d.beta);
    k.alpha = T(d.alpha);
    k.gl = T(d.gamma * d.lambda);
    k.grav = T(d.grav);
    k.rhoref = T(d.rhoref);
    k.itf = T(1.0 / d.tau_f);
    k.itg = T(1.0 / d.tau_g);
    k.pf = T(1.0 - 0.5 / d.tau_f);
    k.pg = T(1.0 - 0.5 / d.tau_g);
    return k;
}

}  // namespace

struct lbm3_sim {
    lbm_params prm;
    lbm::Derived d;
    int nz = 0;
    Layout3 L;
    cudaStream_t stream = nullptr;
    char *state = nullptr, *work = nullptr;
    int cur = 0;
    int64_t steps = 0;
    bool initialized = false;
    std::string err;
    bool f64() const { return prm.dtype == LBM_F64; }
    char *level(int i) const { return state + (size_t)i * L.level; }
    char *field(int i) const { return work + (size_t)i * L.field; }  // 0 phi, 1 mu, 2 p
    double *part() const { return reinterpret_cast<double *>(work + L.part_off); }
    double *out() const { return reinterpret_cast<double *>(work + L.out_off); }
    unsigned blocks() const { return (unsigned)((L.N + kThreads - 1) / kThreads); }
    // step kernels: one row of x per block column, y and z from the grid
    unsigned row_threads() const { return d.nx >= 128 ? 128u : (unsigned)((d.nx + 31) / 32 * 32); }
    dim3 rows() const { return dim3((unsigned)((d.nx + row_threads() - 1) / row_threads()), (unsigned)d.ny, (unsigned)nz); }
    lbm_status fail(lbm_status s, const std::string &m) {
        err = m;
        return s;
    }
    lbm_status cuda(cudaError_t e, const char *what) {
        return e == cudaSuccess ? LBM_OK
                                : fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    lbm_status ready() {
        if (!state || !work) return fail(LBM_ERR_STATE, "buffers not bound");
        return LBM_OK;
    }

    // phi and mu of the current level into the field slots
    template <class T>
    void phi_mu(const K3<T> &P) {
        const T *lvl = reinterpret_cast<const T *>(level(cur));
        lbm3::k3_phi<T><<<rows(), row_threads(), 0, stream>>>(lvl, reinterpret_cast<T *>(field(0)), P);
        lbm3::k3_mu<T><<<rows(), row_threads(), 0, stream>>>(reinterpret_cast<const T *>(field(0)),
                                                           reinterpret_cast<T *>(field(1)), P);
    }
    template <class T>
    void pressure(const K3<T> &P) {
        lbm3::k3_p<T><<<rows(), row_threads(), 0, stream>>>(
            reinterpret_cast<const T *>(level(cur)), reinterpret_cast<const T *>(field(0)),
            reinterpret_cast<const T *>(field(1)), reinterpret_cast<T *>(field(2)), P);
    }
    template <class T>
    lbm_status step_t(int64_t n) {
        const K3<T> P = make_k3<T>(d, nz, L);
        for (int64_t t = 0; t < n; ++t) {
            phi_mu(P);
            pressure(P);
            lbm3::k3_collide<T><<<rows(), row_threads(), 0, stream>>>(
                reinterpret_cast<const T *>(level(cur)), reinterpret_cast<T *>(level(1 - cur)),
                reinterpret_cast<const T *>(field(0)), reinterpret_cast<const T *>(field(1)),
                reinterpret_cast<const T *>(field(2)), P);
            if (lbm_status st = cuda(cudaGetLastError(), "3-D step")) return st;
            cur = 1 - cur;
            ++steps;
        }
        return LBM_OK;
    }
    template <class T>
    lbm_status init_t(const void *phi, const void *ux, const void *uy, const void *uz) {
        const K3<T> P = make_k3<T>(d, nz, L);
        lbm3::k3_mu<T><<<rows(), row_threads(), 0, stream>>>(static_cast<const T *>(phi),
                                                           reinterpret_cast<T *>(field(1)), P);
        lbm3::k3_init<T><<<blocks(), kThreads, 0, stream>>>(
            static_cast<const T *>(phi), reinterpret_cast<const T *>(field(1)),
            static_cast<const T *>(ux), static_cast<const T *>(uy), static_cast<const T *>(uz),
            reinterpret_cast<T *>(level(0)), P);
        return cuda(cudaGetLastError(), "3-D init");
    }
    template <class T>
    lbm_status fields_t(void *phi, void *rho, void *p, void *ux, void *uy, void *uz, void *mu) {
        const K3<T> P = make_k3<T>(d, nz, L);
        phi_mu(P);
        lbm3::k3_fields<T><<<blocks(), kThreads, 0, stream>>>(
            reinterpret_cast<const T *>(level(cur)), reinterpret_cast<const T *>(field(0)),
            reinterpret_cast<const T *>(field(1)), static_cast<T *>(rho), static_cast<T *>(p),
            static_cast<T *>(ux), static_cast<T *>(uy), static_cast<T *>(uz), P);
        if (lbm_status st = cuda(cudaGetLastError(), "3-D fields")) return st;
        const size_t fb = (size_t)L.N * sizeof(T);
        if (phi)
            if (lbm_status st = cuda(cudaMemcpyAsync(phi, field(0), fb, cudaMemcpyDeviceToDevice, stream), "copy phi"))
                return st;
        if (mu)
            if (lbm_status st = cuda(cudaMemcpyAsync(mu, field(1), fb, cudaMemcpyDeviceToDevice, stream), "copy mu"))
                return st;
        return LBM_OK;
    }
    template <class T>
    lbm_status mass_t(double h[2]) {
        const K3<T> P = make_k3<T>(d, nz, L);
        lbm3::k3_mass_partial<T><<<kParts, 256, 0, stream>>>(reinterpret_cast<const T *>(level(cur)),
                                                              part(), P);
        lbm3::k3_fold<<<1, 256, 0, stream>>>(part(), kParts, 2, out());
        if (lbm_status st = cuda(cudaGetLastError(), "3-D mass")) return st;
        if (lbm_status st = cuda(cudaMemcpyAsync(h, out(), 2 * sizeof(double), cudaMemcpyDeviceToHost, stream), "mass copy"))
            return st;
        return cuda(cudaStreamSynchronize(stream), "mass");
    }
    template <class T>
    lbm_status laplace_t(double xc, double yc, double zc, double R, double h[5]) {
        const K3<T> P = make_k3<T>(d, nz, L);
        phi_mu(P);
        pressure(P);
        const double W = prm.W;
        lbm3::k3_laplace_partial<T><<<kParts, 256, 0, stream>>>(
            reinterpret_cast<const T *>(field(0)), reinterpret_cast<const T *>(field(2)), P, d.beta,
            d.kappa, xc, yc, zc, R - 2.0 * W, R + 2.0 * W, part());
        lbm3::k3_fold<<<1, 256, 0, stream>>>(part(), kParts, 5, out());
        if (lbm_status st = cuda(cudaGetLastError(), "3-D laplace")) return st;
        if (lbm_status st = cuda(cudaMemcpyAsync(h, out(), 5 * sizeof(double), cudaMemcpyDeviceToHost, stream), "laplace copy"))
            return st;
        return cuda(cudaStreamSynchronize(stream), "laplace");
    }
};

extern "C" {

lbm_status lbm3_buffer_sizes(const lbm_params *prm, int nz, size_t *state_bytes, size_t *work_bytes) {
    std::string m = check3(prm, nz);
    if (!m.empty()) {
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    const Layout3 L = layout3((long long)prm->nx * prm->ny * nz, prm->dtype == LBM_F64 ? 8 : 4);
    if (state_bytes) *state_bytes = 2 * L.level;
    if (work_bytes) *work_bytes = L.work;
    return LBM_OK;
}

lbm_status lbm3_create(const lbm_params *prm, int nz, void *stream, lbm3_sim **out) {
    if (!out) {
        lbm_internal_set_error("null output pointer");
        return LBM_ERR_ARG;
    }
    *out = nullptr;
    std::string m = check3(prm, nz);
    if (!m.empty()) {
        lbm_internal_set_error(m.c_str());
        return LBM_ERR_ARG;
    }
    lbm3_sim *s = new lbm3_sim();
    s->prm = *prm;
    s->d = lbm::derive(prm);
    s->nz = nz;
    s->L = layout3((long long)prm->nx * prm->ny * nz, prm->dtype == LBM_F64 ? 8 : 4);
    s->stream = static_cast<cudaStream_t>(stream);
    *out = s;
    return LBM_OK;
}

lbm_status lbm3_bind_buffers(lbm3_sim *s, void *state, size_t state_bytes, void *work,
                             size_t work_bytes) {
    if (!s) return LBM_ERR_ARG;
    if (!state || !work) return s->fail(LBM_ERR_ARG, "null buffer");
    if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(work)) & 255)
        return s->fail(LBM_ERR_ARG, "buffers must be 256-byte aligned");
    if (state_bytes < 2 * s->L.level || work_bytes < s->L.work)
        return s->fail(LBM_ERR_NOMEM, "bound buffer smaller than lbm3_buffer_sizes");
    s->state = static_cast<char *>(state);
    s->work = static_cast<char *>(work);
    s->initialized = false;
    return LBM_OK;
}

lbm_status lbm3_init_phi(lbm3_sim *s, const void *phi, const void *ux, const void *uy,
                         const void *uz) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!phi) return s->fail(LBM_ERR_ARG, "phi is null");
    s->cur = 0;
    lbm_status st = s->f64() ? s->init_t<double>(phi, ux, uy, uz) : s->init_t<float>(phi, ux, uy, uz);
    if (st) return st;
    s->steps = 0;
    s->initialized = true;
    return LBM_OK;
}

lbm_status lbm3_step(lbm3_sim *s, int64_t n) {
    if (!s) return LBM_ERR_ARG;
    lbm::NvtxRange r_call("lbm3_step");
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm3_step before lbm3_init_phi");
    if (n < 0) return s->fail(LBM_ERR_ARG, "negative step count");
    return s->f64() ? s->step_t<double>(n) : s->step_t<float>(n);
}

lbm_status lbm3_fields(lbm3_sim *s, void *phi, void *rho, void *p, void *ux, void *uy, void *uz,
                       void *mu) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm3_fields before lbm3_init_phi");
    return s->f64() ? s->fields_t<double>(phi, rho, p, ux, uy, uz, mu)
                    : s->fields_t<float>(phi, rho, p, ux, uy, uz, mu);
}

lbm_status lbm3_mass(lbm3_sim *s, double *mass, double *phi_total) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm3_mass before lbm3_init_phi");
    double h[2];
    lbm_status st = s->f64() ? s->mass_t<double>(h) : s->mass_t<float>(h);
    if (st) return st;
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
        return s->fail(LBM_ERR_NONFINITE, "non-finite mass: the state has diverged");
    if (mass) *mass = h[0];
    if (phi_total) *phi_total = h[1];
    return LBM_OK;
}

lbm_status lbm3_laplace(lbm3_sim *s, double xc, double yc, double zc, double R, double *dP,
                        double *R_eff) {
    if (!s) return LBM_ERR_ARG;
    if (lbm_status st = s->ready()) return st;
    if (!s->initialized) return s->fail(LBM_ERR_STATE, "lbm3_laplace before lbm3_init_phi");
    double h[5];
    lbm_status st = s->f64() ? s->laplace_t<double>(xc, yc, zc, R, h)
                             : s->laplace_t<float>(xc, yc, zc, R, h);
    if (st) return st;
    if (dP) *dP = (h[1] > 0 ? h[0] / h[1] : 0.0) - (h[3] > 0 ? h[2] / h[3] : 0.0);
    if (R_eff) *R_eff = std::cbrt(3.0 * h[4] / (4.0 * 3.14159265358979323846));
    return LBM_OK;
}

int64_t lbm3_step_count(const lbm3_sim *s) { return s ? s->steps : 0; }

const char *lbm3_last_error(const lbm3_sim *s) { return s ? s->err.c_str() : "null handle"; }

void lbm3_destroy(lbm3_sim *s) { delete s; }

}  // extern "C"
