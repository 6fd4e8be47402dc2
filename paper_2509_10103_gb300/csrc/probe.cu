// Measured FMA throughput of the device (FP64 or FP32), the denominator of
// the ALU roofline that the library's FP64-bound kernels are judged against.
// A GB300 runs FP64 at 1/64 of its FP32 rate, so its FP64 roof is far from
// any datasheet "tensor" figure and is measured here instead of assumed.
//
// Every thread runs kAcc independent fma chains x <- x a + b (a slightly
// below 1, so the values stay bounded) for `iters` iterations; a grid of
// kBlocksPerSM blocks of 256 threads per SM keeps every FMA lane busy.  The
// chains' sum is compared with a value it never takes, so the compiler keeps
// every FMA; the result is never stored in practice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/pnop.h"

namespace {

constexpr int kAcc = 8, kThreads = 256, kBlocksPerSM = 8;

__device__ double g_probe_sink;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T a, T b) {
    T x[kAcc];
#pragma unroll
    for (int i = 0; i < kAcc; ++i) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kAcc; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kAcc; ++i) s += x[i];
    if (s == (T)-1.0) g_probe_sink = (double)s;
}

template <class T>
int measure(int iters, int blocks, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PNOP_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PNOP_ERR_CUDA;
    }
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.9999999, (T)1e-7);
    cudaEventRecord(e1, s);
    int rc = PNOP_OK;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        rc = PNOP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

template <class T>
int peak(double seconds, cudaStream_t s, double* tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PNOP_ERR_CUDA;
    const int blocks = nsm * kBlocksPerSM;
    float ms = 0;
    int iters = 1024;
    int rc = measure<T>(iters, blocks, s, &ms);  // warm-up and calibration
    if (rc != PNOP_OK) return rc;
    // scale to about `seconds` per launch, in bounds: at most 2^26 iterations
    const double want = std::max(1e-3, seconds) * 1e3;
    const double scale = ms > 0 ? want / ms : 64.0;
    iters = (int)std::min(67108864.0, std::max(1024.0, iters * scale));
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        rc = measure<T>(iters, blocks, s, &ms);
        if (rc != PNOP_OK) return rc;
        const double flops = 2.0 * kAcc * (double)iters * (double)blocks * kThreads;
        if (ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    *tflops = best;
    return best > 0 ? PNOP_OK : PNOP_ERR_CUDA;
}

}  // namespace

extern "C" int pnop_measure_fma_peak(int precision, double seconds, void* cuda_stream, double* tflops) {
    if (!tflops || !(seconds > 0) || seconds > 10 || (precision != PNOP_FP64 && precision != PNOP_MIXED))
        return PNOP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return precision == PNOP_FP64 ? peak<double>(seconds, s, tflops) : peak<float>(seconds, s, tflops);
}
