// Device helpers shared by the kernel translation units: complex arithmetic in
// FP64 or FP32, precision conversion, launch checks.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <stdexcept>

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

// FP64 <-> FP32 conversions on the integer pipes, from the IEEE-754 binary64
// and binary32 layouts: the FP64 pipe of this GPU issues two lanes per SM per
// cycle, so the conversion instructions it would execute dominate the FP32
// transform kernels.  Round to nearest even, infinities and NaNs kept; the
// rare values below the smallest normal float (|x| < 2^-126) take the
// hardware conversion.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // upper 23 of the 52 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                   // the 29 bits dropped
    const int fe = e - 1023 + 127;
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | m | ((m | rest) ? 0x400000u : 0u));
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    if (fe <= 0) return (float)x;
    unsigned r = sign | ((unsigned)fe << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;  // carries into the exponent as it should
    return __uint_as_float(r);
}
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0) return (double)f;
    const unsigned de = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
    return __hiloint2double((int)(sign | (de << 20) | (m >> 3)), (int)(m << 29));
}

template <class T2> __device__ __forceinline__ T2 from_d(double2 v);
template <> __device__ __forceinline__ double2 from_d<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d<float2>(double2 v) { return make_float2(d2f_rn(v.x), d2f_rn(v.y)); }
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(f2d_exact(v.x), f2d_exact(v.y)); }

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

}  // namespace pnop
