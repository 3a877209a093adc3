// FP32 FMA throughput of the GPU, measured: the denominator of the roofline
// that the DP kernels (bound by FP32 lane arithmetic, not by HBM) are
// reported against.
//
// Every thread runs 8 independent chains x = fma(x, a, b), 16 per chain per
// loop trip (128 FFMA), so each warp always has independent FMAs to issue;
// two CTAs of 1024 threads per SM keep 16 warps on every SM sub-partition.
// a and b are kernel arguments, so the compiler cannot fold the chains; the
// result is stored only when it equals a value the chains never reach
// (a < 1 keeps them bounded), which keeps the loop alive without traffic.
#include <cuda_runtime.h>

#include <algorithm>

#include "pardtw_common.cuh"

namespace pardtw {
namespace {

constexpr int kPeakThreads = 1024;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads, 2)
    k_ffma_peak(float* __restrict__ sink, int iters, float a, float b) {
    float x[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += x[c];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace pardtw

using namespace pardtw;

extern "C" int dtw_fp32_peak(int device, int iters, double* ffma_per_s) {
    if (!ffma_per_s || iters < 1) return DTW_ERR_INVALID;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return DTW_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_INVALID;
    }
    int rc = DTW_OK;
    int sms = 0;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&sink, (size_t)2 * sms * kPeakThreads * sizeof(float)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DTW_ERR_CUDA;
    } else {
        const unsigned grid = (unsigned)(2 * sms);
        k_ffma_peak<<<grid, kPeakThreads>>>(sink, iters / 4 + 1, 0.9999f, 1e-4f);  // warm-up
        for (int rep = 0; rep < 3 && rc == DTW_OK; ++rep) {
            float ms = 0.f;
            if (cudaEventRecord(e0) != cudaSuccess) rc = DTW_ERR_CUDA;
            k_ffma_peak<<<grid, kPeakThreads>>>(sink, iters, 0.9999f, 1e-4f);
            if (rc == DTW_OK && (cudaGetLastError() != cudaSuccess ||
                                 cudaEventRecord(e1) != cudaSuccess ||
                                 cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f))
                rc = DTW_ERR_CUDA;
            if (rc == DTW_OK) {
                const double ffma = (double)grid * kPeakThreads * iters * kPeakChains * kPeakUnroll;
                best = std::max(best, ffma / (ms * 1e-3));
            }
        }
    }
    if (rc != DTW_OK) (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    *ffma_per_s = best;
    return rc;
}
