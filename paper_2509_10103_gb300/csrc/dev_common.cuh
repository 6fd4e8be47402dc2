// Device helpers shared by the kernel translation units: complex arithmetic in
// FP64 or FP32, precision conversion, launch checks.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <set>
#include <stdexcept>
#include <utility>

namespace pnop {

constexpr int kB = 13;  // stored band (columns j-4 .. j+8)

// ------------------------------------------------------------------ complex helpers
template <class T2> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <class T2>
__device__ __forceinline__ T2 mk(typename RealOf<T2>::T x, typename RealOf<T2>::T y) {
    T2 r;
    r.x = x;
    r.y = y;
    return r;
}
template <class T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk<T2>(a.x + b.x, a.y + b.y); }
template <class T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk<T2>(a.x - b.x, a.y - b.y); }
template <class T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk<T2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// s * i * z
template <class T2> __device__ __forceinline__ T2 imul(T2 z, typename RealOf<T2>::T s) { return mk<T2>(-s * z.y, s * z.x); }
__device__ __forceinline__ double2 dscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 dfma(double s, double2 a, double2 acc) {
    return make_double2(fma(s, a.x, acc.x), fma(s, a.y, acc.y));
}

// FP32 -> FP64 conversion by integer operations on the bit pattern (exact).
// The GB300's FP64 pipe, which also executes the hardware conversions, runs at
// 1/64 of the FP32 rate, and the mixed-precision theta analysis converts every
// spectral value it writes; this takes integer issue slots instead.  Zero and
// subnormals become signed zero; infinities and NaN stay infinite and NaN (so
// that a non-finite field is still detected).
__device__ __forceinline__ double f64_of(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0) return __longlong_as_double((long long)sign);  // zero (subnormals flushed)
    const unsigned long long de = e == 0xFFu ? 0x7FFull : (unsigned long long)e + 896ull;
    return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

template <class T2> __device__ __forceinline__ T2 from_d(double2 v);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 v) { return v; }
// The theta synthesis converts with the hardware (its FP64 pipe has room
// between the loads), the theta analysis by integer operations (its FP64 pipe
// also carries the additions of the base-flow terms): each measured fastest
// that way on the 64x64x256 gradient.
template <> __device__ __forceinline__ float2 from_d<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(f64_of(v.x), f64_of(v.y)); }

__device__ __forceinline__ int par_idx(int m) { return m & 1; }  // 0 even, 1 odd (two's complement)

// scale factor of the transform precision (no FP64->FP32 conversion in FP32 kernels)
template <class T> __device__ __forceinline__ T zs(const double* d, const float* f, int i);
template <> __device__ __forceinline__ double zs<double>(const double* d, const float*, int i) { return d[i]; }
template <> __device__ __forceinline__ float zs<float>(const double*, const float* f, int i) { return f[i]; }

static inline void check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
        throw std::runtime_error(buf);
    }
}
static inline unsigned nblk(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------------ launches
// Programmatic dependent launch.  Every kernel of the library starts with
// grid_dep_sync(): it waits until the grids it depends on have completed and
// their writes are visible, then allows the next grid on the stream to be
// launched at once.  A kernel launched with launch_pdl can thus be scheduled
// while its predecessor is still in its last wave, and starts work the moment
// the predecessor ends, instead of after a full launch round trip; it never
// reads or writes memory before the wait, so stream order is kept.
// launch_serial launches without that relaxation: the single-wave kernels
// whose time depends on an even spread of their blocks over the SMs (the
// banded solves) use it, so that all their blocks are placed on an idle GPU.
__device__ __forceinline__ void grid_dep_sync() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class... KArgs, class... Args>
inline void launch_serial(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raises the dynamic shared-memory limit of a kernel to 200 KB once per
// (kernel, device): the attribute is per device, and launches come from
// several host threads (the serving layer) and several devices.
inline void smem_limit(const void* kernel) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.insert({kernel, dev}).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace pnop
