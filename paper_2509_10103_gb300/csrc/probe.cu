// Measured FMA throughput of the device (FP64 or FP32), the denominator of
// the ALU roofline that the library's FP64-bound kernels are judged against.
// A GB300 runs FP64 at 1/64 of its FP32 rate, so its FP64 roof is far from
// any datasheet "tensor" figure and is measured here instead of assumed.
//
// Every thread runs ACC independent fma chains x <- x a + b (a slightly
// below 1, so the values stay bounded) for `iters` iterations, on a grid of a
// few blocks of 256 threads per SM.  The chains' sum is compared with a value
// it never takes, so the compiler keeps every FMA; the result is never stored
// in practice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/pnop.h"

namespace {

constexpr int kThreads = 256;

__device__ double g_probe_sink;

template <class T, int ACC>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T a, T b) {
    T x[ACC];
#pragma unroll
    for (int i = 0; i < ACC; ++i) x[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < ACC; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < ACC; ++i) s += x[i];
    if (s == (T)-1.0) g_probe_sink = (double)s;
}

template <class T, int ACC>
int measure(int iters, int blocks, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PNOP_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PNOP_ERR_CUDA;
    }
    cudaEventRecord(e0, s);
    k_fma_probe<T, ACC><<<blocks, kThreads, 0, s>>>(iters, (T)0.9999999, (T)1e-7);
    cudaEventRecord(e1, s);
    int rc = PNOP_OK;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        rc = PNOP_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Best rate of one configuration (ACC chains per thread, bps blocks per SM):
// calibrate to about `seconds` per launch, then the best of three launches.
template <class T, int ACC>
int peak_of(double seconds, int nsm, int bps, cudaStream_t s, double* best) {
    const int blocks = nsm * bps;
    float ms = 0;
    int iters = 1024;
    int rc = measure<T, ACC>(iters, blocks, s, &ms);  // warm-up and calibration
    if (rc != PNOP_OK) return rc;
    const double want = std::max(1e-3, seconds) * 1e3;
    const double scale = ms > 0 ? want / ms : 64.0;
    iters = (int)std::min(67108864.0, std::max(1024.0, iters * scale));  // in bounds: at most 2^26
    for (int rep = 0; rep < 3; ++rep) {
        rc = measure<T, ACC>(iters, blocks, s, &ms);
        if (rc != PNOP_OK) return rc;
        const double flops = 2.0 * ACC * (double)iters * (double)blocks * kThreads;
        if (ms > 0) *best = std::max(*best, flops / (ms * 1e-3) / 1e12);
    }
    return PNOP_OK;
}

// The FMA pipes are full only with enough independent chains per scheduler;
// how many are needed depends on the pipe's latency and width, so a few
// chain counts and occupancies are tried and the best rate is the peak.
template <class T>
int peak(double seconds, cudaStream_t s, double* tflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PNOP_ERR_CUDA;
    double best = 0;
    for (int bps : {2, 4, 8}) {
        int rc = peak_of<T, 4>(seconds, nsm, bps, s, &best);
        if (rc == PNOP_OK) rc = peak_of<T, 8>(seconds, nsm, bps, s, &best);
        if (rc == PNOP_OK) rc = peak_of<T, 16>(seconds, nsm, bps, s, &best);
        if (rc != PNOP_OK) return rc;
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
