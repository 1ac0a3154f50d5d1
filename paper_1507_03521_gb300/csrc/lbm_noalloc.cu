// lbm_noalloc.cu — the mass diagnostic for callers that cannot allocate
// device memory.
//
// lbm_mass needs a handle with a caller-allocated work buffer, which holds
// the reduction's per-block partial sums.  Some callers cannot provide one:
// host programs whose device memory is a fixed budget handed out by
// someone else, plug-ins that must not change the process's device
// footprint, and loops that cannot afford cudaMalloc's implicit device-wide
// synchronisation.  They still hold the populations, and they want the
// same two numbers.  lbm_mass_noalloc gives them those numbers with no
// handle and no allocation: its scratch is the file-scope device array
// below, loaded with this library and kept until the process exits.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_ops.cuh"

namespace {

// The scratch holds the partial sums of at most kMaxBlocks blocks.  A block
// reduces `span` cells: N / kMaxBlocks rounded up to a multiple of 256, but
// at least kMinSpan, so that mid-size grids still spread over many blocks
// (a 2048 x 2048 grid gets 1024).  Spans are capped at kMaxSpan, which
// limits grids to 2^28 cells (16384 x 16384).  2 * 4096 + 2 doubles = 64 KB
// + 16 B per device.
constexpr int kMaxBlocks = 4096;
constexpr long long kMinSpan = 4096, kMaxSpan = 65536;
constexpr long long kMaxCells = (long long)kMaxBlocks * kMaxSpan;
constexpr int kScratchDoubles = 2 * kMaxBlocks + 2;

long long block_span(long long N) {
    long long span = (N + kMaxBlocks - 1) / kMaxBlocks;
    span = (span + 255) / 256 * 256;
    return span < kMinSpan ? kMinSpan : span;
}

// Per-block partials at [2b, 2b + 1]; the final sums at [2 kMaxBlocks, +1].
// Every slot a call reads is written earlier in the same call, so nothing
// has to be cleared between calls; the contents of the last call stay.
static __device__ __align__(256) double g_mass_scratch[kScratchDoubles];

template <class T, class ST>
__global__ void __launch_bounds__(256)
k_mass_noalloc_partial(const char *__restrict__ lvl, const lbm::KP<T> P, long long span,
                       double *__restrict__ scratch) {
    const long long N = (long long)P.nx * P.ny;
    const long long b0 = (long long)blockIdx.x * span;
    const long long b1 = b0 + span < N ? b0 + span : N;
    const double rhoB = (double)P.rhoB, phiB = (double)P.phiB, drho = (double)P.drho;
    double sm = 0.0, sp = 0.0;
    for (long long k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
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
        scratch[2 * blockIdx.x] = a;
        scratch[2 * blockIdx.x + 1] = b;
    }
}

// Sums the per-block partials in block order into the two final slots.
__global__ void k_mass_noalloc_final(int nblocks, double *__restrict__ scratch) {
    if (threadIdx.x < 2) {
        double a = 0.0;
        for (int b = 0; b < nblocks; ++b) a += scratch[2 * b + threadIdx.x];
        scratch[2 * kMaxBlocks + threadIdx.x] = a;
    }
}

// Device address of g_mass_scratch for the current device.  In host code
// the name g_mass_scratch is only a host-side stand-in, not a device
// address, so it is looked up with cudaGetSymbolAddress, on every call: the
// lookup is cheap next to the two launches and the synchronisation, and a
// cached address would go stale if the module were reloaded (after a
// cudaDeviceReset).
lbm_status scratch_address(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mass_scratch);
    if (e != cudaSuccess || !p) {
        lbm_internal_set_error("lbm_mass_noalloc: cudaGetSymbolAddress failed");
        return LBM_ERR_CUDA;
    }
    *out = static_cast<double *>(p);
    return LBM_OK;
}

template <class T, class ST>
cudaError_t launch(const lbm::Derived &d, const void *level, double *scratch, long long span,
                   int nblocks, cudaStream_t s) {
    k_mass_noalloc_partial<T, ST><<<nblocks, 256, 0, s>>>(static_cast<const char *>(level),
                                                          lbm::make_kp<T>(d), span, scratch);
    k_mass_noalloc_final<<<1, 32, 0, s>>>(nblocks, scratch);
    return cudaGetLastError();
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const lbm_params *prm, const void *level, void *stream,
                                       double *mass, double *phi_total) {
    // Parameter validation is the one lbm_buffer_sizes applies (host only).
    if (lbm_status st = lbm_buffer_sizes(prm, nullptr, nullptr)) return st;
    if (!level) {
        lbm_internal_set_error("lbm_mass_noalloc: level is null");
        return LBM_ERR_ARG;
    }
    const long long N = (long long)prm->nx * prm->ny;
    if (N > kMaxCells) {
        lbm_internal_set_error(
            "lbm_mass_noalloc: grid exceeds the static scratch limit of 268435456 cells "
            "(2^28, e.g. 16384 x 16384); use lbm_mass with a bound work buffer");
        return LBM_ERR_NOMEM;
    }
    double *scratch = nullptr;
    if (lbm_status st = scratch_address(&scratch)) return st;

    lbm::Derived d{};
    d.nx = prm->nx;
    d.ny = prm->ny;
    d.N = N;
    d.NS = (N + 127) / 128 * 128;  // slot stride of the library's level layout
    d.phiB = prm->phi_B;
    d.rhoB = prm->rho_B;
    d.drho = (prm->rho_A - prm->rho_B) / (prm->phi_A - prm->phi_B);  // Eq. 13
    d.tau_f = prm->tau_f;
    d.tau_g = prm->tau_g;

    const long long span = block_span(N);
    const int nblocks = (int)((N + span - 1) / span);  // <= kMaxBlocks for N <= kMaxCells
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (prm->dtype) {
        case LBM_F64: e = launch<double, lbm::PlainStore<double>>(d, level, scratch, span, nblocks, s); break;
        case LBM_F32: e = launch<float, lbm::PlainStore<float>>(d, level, scratch, span, nblocks, s); break;
        case LBM_F16S: e = launch<float, lbm::Store16<__half>>(d, level, scratch, span, nblocks, s); break;
        case LBM_BF16S: e = launch<float, lbm::Store16<__nv_bfloat16>>(d, level, scratch, span, nblocks, s); break;
        case LBM_F16D: e = launch<float, lbm::Store16D<__half>>(d, level, scratch, span, nblocks, s); break;
        default: e = launch<float, lbm::Store16D<__nv_bfloat16>>(d, level, scratch, span, nblocks, s); break;
    }
    double h[2] = {0.0, 0.0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch + 2 * kMaxBlocks, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        lbm_internal_set_error(cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (mass) *mass = h[0];
    if (phi_total) *phi_total = h[1];
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
        lbm_internal_set_error("lbm_mass_noalloc: non-finite mass or phi total");
        return LBM_ERR_NONFINITE;
    }
    return LBM_OK;
}
