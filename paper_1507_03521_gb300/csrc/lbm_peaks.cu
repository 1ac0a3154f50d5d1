// lbm_peaks.cu — the GPU's measured FMA throughput (FP32 scalar, FP32
// packed pairs, FP64), the ALU ceiling that the step's arithmetic is held
// against.  Not part of the method: a measurement aid of the library.
//
// Each thread runs 8 independent chains x <- x a + b (a just below 1, so
// every chain stays near b / (1 - a) and never overflows or goes
// subnormal), enough independent work per warp to keep the FMA pipe busy.
// The grid is 16 CTAs of 256 threads per SM.  One untimed launch warms the
// clocks; the second is timed with CUDA events on a stream of its own.
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 16;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T *sink, T a, T b, int iters) {
    T x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x % 7) + T(j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == T(-1)) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(kThreads) k_fma2_chains(float *sink, float a, float b, int iters) {
    float2 x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = make_float2(float(threadIdx.x % 7) + j, float(j) - 1.0f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
    if (s == -1.0f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" {

lbm_status lbm_alu_peak(int kind, double *fma_per_s) {
    if (!fma_per_s || kind < 0 || kind > 2) return LBM_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_ERR_CUDA;
    const int blocks = sms * kBlocksPerSM;
    const int iters = kind == 2 ? 2048 : 16384;
    void *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lbm_status rc = LBM_ERR_CUDA;
    float ms = 0.f;
    if (cudaMalloc(&sink, kThreads * sizeof(double)) != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        if (kind == 0)
            k_fma_chains<float><<<blocks, kThreads, 0, st>>>(static_cast<float *>(sink), 0.999f, 1e-3f, iters);
        else if (kind == 1)
            k_fma2_chains<<<blocks, kThreads, 0, st>>>(static_cast<float *>(sink), 0.999f, 1e-3f, iters);
        else
            k_fma_chains<double><<<blocks, kThreads, 0, st>>>(static_cast<double *>(sink), 0.999, 1e-3, iters);
        if (rep == 1) cudaEventRecord(e1, st);
    }
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        goto done;
    {
        // FMA operations: one per chain step, two per packed step
        const double ops = (double)blocks * kThreads * kChains * iters * (kind == 1 ? 2.0 : 1.0);
        *fma_per_s = ops / (ms * 1e-3);
    }
    rc = LBM_OK;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return rc;
}

}  // extern "C"
