// Measured arithmetic peaks: the denominators of the FP32- and FP64-pipe
// rooflines of the solve's kernels (M2L and P2P run on the FP32 pipe in
// mixed precision, on the FP64 pipe in FP64 mode).
//
// Every thread runs kChains independent fused multiply-add chains
// x <- x * a + b, kUnroll deep per loop trip, so each warp always has
// independent FMAs to issue; a full grid (kBlocksPerSM blocks of 256 threads
// per SM) keeps every scheduler busy. a = 1 - 2^-20 and b = 2^-24 keep the
// values near b / (1 - a) = 1/16, far from denormals and overflow. One FMA
// counts as two flops.
#include <algorithm>

#include "gbfmm_internal.cuh"

namespace gbfmm {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* __restrict__ sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-4);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // never true for these a and b; the store keeps the chains alive
    if (s < T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_chains(int iters, T* sink, cudaStream_t st, double* ms) {
    const int grid = device_sm_count() * kBlocksPerSM;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FMM_ERR_CUDA;
    }
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 16777216.0);
    cudaEventRecord(e0, st);
    (k_fma_chains<T><<<grid, kThreads, 0, st>>>(sink, iters, a, b), note_launch());
    cudaEventRecord(e1, st);
    const cudaError_t rc = cudaEventSynchronize(e1);
    float t = 0.f;
    if (rc == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != cudaSuccess || cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    *ms = t;
    return FMM_OK;
}

template <typename T>
int fma_peak(double target_ms, double* tflops, cudaStream_t st) {
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * (size_t)device_sm_count() * kBlocksPerSM * kThreads) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ERR_OOM;
    }
    int iters = 64, rc = FMM_OK;
    double ms = 0.0;
    // grow the loop until one launch lasts about target_ms (clocks settle), then time three
    for (int k = 0; k < 24; ++k) {
        if ((rc = time_chains<T>(iters, sink, st, &ms)) != FMM_OK) break;
        if (ms >= 0.5 * target_ms || iters > (1 << 26)) break;
        const double grow = ms > 0.05 ? target_ms / ms : 16.0;
        iters = (int)std::min<double>((double)iters * std::min(grow, 16.0), (double)(1 << 27));
    }
    double best = 1e30;
    for (int k = 0; rc == FMM_OK && k < 3; ++k) {
        rc = time_chains<T>(iters, sink, st, &ms);
        best = ms < best ? ms : best;
    }
    cudaFree(sink);
    if (rc != FMM_OK) return rc;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * device_sm_count() * kBlocksPerSM * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return FMM_OK;
}

}  // namespace
}  // namespace gbfmm

using namespace gbfmm;

extern "C" int fmm_fma_peak(int precision, double target_ms, double* tflops, void* cuda_stream) {
    if (!tflops || !(target_ms > 0.0) || target_ms > 10000.0 ||
        (precision != FMM_PRECISION_FP64 && precision != FMM_PRECISION_MIXED)) {
        set_global_error("fmm_fma_peak: precision must be FMM_PRECISION_FP64 or FMM_PRECISION_MIXED (FP32), "
                         "target_ms in (0, 10000], tflops non-NULL");
        return FMM_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int rc = precision == FMM_PRECISION_FP64 ? fma_peak<double>(target_ms, tflops, st)
                                                   : fma_peak<float>(target_ms, tflops, st);
    if (rc != FMM_OK) set_global_error("fmm_fma_peak: a CUDA call failed");
    return rc;
}
