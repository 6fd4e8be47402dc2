// Double-float ("double-FP32") arithmetic for the explicit banded products
// of the radial stage and the curl: a value is the unevaluated sum hi + lo of
// two floats, about 48 significant bits.  Products are made exact with an FMA
// (Dekker 1971, "A floating-point technique for extending the available
// precision"; Knuth's two-sum for the additions), so a 9-point band row keeps
// its cancellation under control at FP32 issue rates.  On a GPU whose FP64
// rate is 1/64 of its FP32 rate this trades one FP64 instruction for about a
// dozen FP32 and integer ones.
//
// Conversions avoid the FP64 pipe: a double is split into its significand
// truncated to 24 bits (hi) and the remaining 29 bits rounded to a float (lo)
// by integer operations on its bit pattern, and a pair is joined back by
// rebuilding each float as a double bit pattern and one FP64 addition.
// Magnitudes below 2^-74 lose their lo part (relative error 2^-23 there) and
// below 2^-126 are flushed to zero; the fields this is used on are far above
// that.
#pragma once

#include <cuda_runtime.h>

namespace pnop {

struct dfl {
    float h, l;
};
struct dfc {  // complex double-float
    dfl re, im;
};

// x = hi + lo with hi its significand truncated to 24 bits
__device__ __forceinline__ dfl df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7FFu);
    dfl r;
    if (e <= 896) {  // |x| < 2^-126 (zero included): flushed
        r.h = 0.f;
        r.l = 0.f;
        return r;
    }
    const unsigned sign = hw & 0x80000000u;
    r.h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hw & 0x000FFFFFu) << 3) | (lw >> 29));
    const unsigned rem = lw & 0x1FFFFFFFu;  // value rem * 2^(e - 1075), the sign of x
    if (e >= 949 && rem) {
        const float scale = __uint_as_float((unsigned)(e - 948) << 23);
        r.l = __uint_as_float(__float_as_uint((float)rem * scale) | sign);
    } else {
        r.l = 0.f;
    }
    return r;
}

// a float as a double, by its bit pattern (normal floats and zero)
__device__ __forceinline__ double df_f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if ((u & 0x7F800000u) == 0) return __longlong_as_double((long long)sign);  // zero (and flushed subnormals)
    const unsigned long long e = ((u >> 23) & 0xFFu) + 896ull;
    return __longlong_as_double((long long)(sign | (e << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ double df_join(dfl a) { return df_f2d(a.h) + df_f2d(a.l); }

__device__ __forceinline__ dfc df_load(const double2* p) {
    const double2 v = *p;
    dfc r;
    r.re = df_split(v.x);
    r.im = df_split(v.y);
    return r;
}
__device__ __forceinline__ double2 df_join2(const dfc& a) { return make_double2(df_join(a.re), df_join(a.im)); }

// accumulator (s, c): running sum s and its collected error terms c
struct dacc {
    float s, c;
};
__device__ __forceinline__ dacc dacc0() {
    dacc a;
    a.s = 0.f;
    a.c = 0.f;
    return a;
}
// a += k x, k and x double-floats: the product of the high parts exactly
// (FMA), its cross terms, and the sum's rounding error (two-sum) go to a.c
__device__ __forceinline__ void df_fma(dacc& a, dfl k, dfl x) {
    const float p = k.h * x.h;
    float e = fmaf(k.h, x.h, -p);
    e = fmaf(k.h, x.l, e);
    e = fmaf(k.l, x.h, e);
    const float s = a.s + p;
    const float bb = s - a.s;
    const float err = (a.s - (s - bb)) + (p - bb);
    a.s = s;
    a.c += err + e;
}
// a += x (a double-float)
__device__ __forceinline__ void df_add(dacc& a, dfl x) {
    const float s = a.s + x.h;
    const float bb = s - a.s;
    const float err = (a.s - (s - bb)) + (x.h - bb);
    a.s = s;
    a.c += err + x.l;
}
__device__ __forceinline__ dfl df_neg(dfl x) {
    x.h = -x.h;
    x.l = -x.l;
    return x;
}
// the accumulated value as a normalised pair
__device__ __forceinline__ dfl df_val(dacc a) {
    dfl r;
    r.h = a.s + a.c;
    r.l = a.c - (r.h - a.s);
    return r;
}
__device__ __forceinline__ double df_result(dacc a) { return df_join(df_val(a)); }

}  // namespace pnop
