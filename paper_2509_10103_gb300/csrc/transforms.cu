// Spectral <-> physical transforms of the pseudo-spectral pipe-flow step
// (Keuchel & Avila, Section 2.4): theta synthesis, the z pass with the
// pointwise products of the nonlinear term, theta analysis.  3/2-padded grids,
// hand-written shared-memory FFTs templated on FP64 or FP32.  Batched launches
// carry the batch entry in the grid's z dimension (with the field index for
// the theta kernels) and offset spectral and physical buffers by its slot.
#include "dev_common.cuh"
#include "kernels.hpp"

#include <algorithm>
#include <type_traits>
#include <utility>

namespace pnop {

// ------------------------------------------------------------------ shared-memory FFT
// Batched Stockham FFT (autosort) over `ncol` columns of length N stored as
// a[n * ld + col].  Radix 4, then 2, then 3 stages; N = 2^p 3^q.  tw holds
// e^{-2 pi i n / N}; sign = -1 forward, +1 inverse (unnormalised).  Returns the
// buffer holding the result.  All threads of the block must call it.
template <class T2>
__device__ __forceinline__ void small_dft(T2* v, const int R, const int sign) {
    using T = typename RealOf<T2>::T;
    if (R == 2) {
        T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        T2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        T2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        T2 id = imul(d13, (T)sign);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, id);
        v[3] = csub(d02, id);
    } else {  // R == 3
        const T h = (T)0.86602540378443864676;  // sqrt(3)/2
        T2 t1 = cadd(v[1], v[2]);
        T2 t2 = mk<T2>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        T2 d = csub(v[1], v[2]);
        T2 t3 = imul(d, (T)sign * h);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
}

// One radix-R Stockham stage.  Ns (the size of the sub-transforms already
// done) is a power of two 2^lgNs for every stage but the second and later
// radix-3 stages (radix 3 runs last), so the index split is a shift there.
template <class T2, int R, int NCOL, int LD, int SIGN>
__device__ __forceinline__ void fft_stage(const T2* __restrict__ a, T2* __restrict__ b, int N, int Ns, int lgNs,
                                          const T2* __restrict__ tw) {
    const int stride = N / R;
    const int nb = stride * NCOL;
    const int tstep = N / (Ns * R);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int col = idx % NCOL;
        const int jb = idx / NCOL;
        int q, kk;
        if (lgNs >= 0) {
            q = jb >> lgNs;
            kk = jb & (Ns - 1);
        } else {
            q = jb / Ns;
            kk = jb - q * Ns;
        }
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = a[(jb + r * stride) * LD + col];
        if (Ns > 1) {  // the first stage has unit twiddles
            const int tb = kk * tstep;  // r * tb < N
#pragma unroll
            for (int r = 1; r < R; ++r) {
                T2 w = tw[r * tb];
                if (SIGN > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        small_dft(v, R, SIGN);
        const int idxD = q * Ns * R + kk;
#pragma unroll
        for (int r = 0; r < R; ++r) b[(idxD + r * Ns) * LD + col] = v[r];
    }
}

template <class T2, int NCOL, int LD, int SIGN>
__device__ T2* fft_cols(T2* a, T2* b, int N, const T2* tw) {
    const int n2 = __ffs(N) - 1;  // N = 2^n2 3^n3
    int n3 = 0;
    for (int t = N >> n2; t > 1; t /= 3) ++n3;
    int Ns = 1, lgNs = 0;
    for (int st = 0; st < n2 / 2; ++st) {
        fft_stage<T2, 4, NCOL, LD, SIGN>(a, b, N, Ns, lgNs, tw);
        __syncthreads();
        T2* t = a; a = b; b = t;
        Ns *= 4;
        lgNs += 2;
    }
    if (n2 & 1) {
        fft_stage<T2, 2, NCOL, LD, SIGN>(a, b, N, Ns, lgNs, tw);
        __syncthreads();
        T2* t = a; a = b; b = t;
        Ns *= 2;
        lgNs += 1;
    }
    for (int st = 0; st < n3; ++st) {
        fft_stage<T2, 3, NCOL, LD, SIGN>(a, b, N, Ns, st == 0 ? lgNs : -1, tw);
        __syncthreads();
        T2* t = a; a = b; b = t;
        Ns *= 3;
    }
    return a;
}

// spectral input value of a synthesis: fields stored in FP32 (FieldPtrs::inf)
// are read as they are, FP64 fields converted to the transform precision
template <class T2> __device__ __forceinline__ T2 from_f(float2 v);
template <> __device__ __forceinline__ float2 from_f<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 from_f<double2>(float2 v) { return to_d(v); }
// an analysis result for an FP32 output field (FP64 transforms round it)
__device__ __forceinline__ float2 to_f(float2 v) { return v; }
__device__ __forceinline__ float2 to_f(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <class T2>
__device__ __forceinline__ T2 synth_in(const double2* src, const float2* srcf, size_t i) {
    return srcf ? from_f<T2>(srcf[i]) : from_d<T2>(src[i]);
}

// ------------------------------------------------------------------ theta synthesis
// Y[f][j][a][k] = sum_m X_f[j][m][k] e^{i m theta_a}   (zero-padded to nt points)
template <class T2, int KB>
__global__ void k_synth_theta(Geo g, FieldPtrs f, T2* __restrict__ Y, const T2* __restrict__ twg) {
    grid_dep_sync();
    extern __shared__ __align__(16) unsigned char smem[];
    T2* buf0 = reinterpret_cast<T2*>(smem);
    T2* buf1 = buf0 + g.nt * KB;
    T2* tw = buf1 + g.nt * KB;
    const int k0 = blockIdx.x * KB, j = blockIdx.y;
    const int nf = gridDim.z / g.nb, b = blockIdx.z / nf, fi = blockIdx.z - b * nf, slot = g.slot[b];
    Y += (size_t)slot * g.ps;
    const int kw = min(KB, g.nk - k0);
    for (int i = threadIdx.x; i < g.nt; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < g.nt * KB; i += blockDim.x) buf0[i] = mk<T2>(0, 0);
    __syncthreads();
    const size_t base = (size_t)slot * g.fs + (size_t)j * g.nm * g.nk;
    const float2* srcf = f.inf[fi] ? f.inf[fi] + base : nullptr;
    const double2* src = srcf ? nullptr : f.in[fi] + base;
    for (int i = threadIdx.x; i < g.nm * KB; i += blockDim.x) {
        const int im = i / KB, kk = i % KB;
        if (kk < kw) {
            const int m = im - g.M;
            const int a = m < 0 ? m + g.nt : m;
            buf0[a * KB + kk] = synth_in<T2>(src, srcf, (size_t)im * g.nk + k0 + kk);
        }
    }
    __syncthreads();
    T2* res = fft_cols<T2, KB, KB, +1>(buf0, buf1, g.nt, tw);
    T2* dst = Y + ((size_t)(fi * g.nr + j) * g.nt) * g.nk;
    for (int i = threadIdx.x; i < g.nt * KB; i += blockDim.x) {
        const int a = i / KB, kk = i % KB;
        if (kk < kw) dst[(size_t)a * g.nk + k0 + kk] = res[i];
    }
}

// Products of the continuous-adjoint forcing at one physical point from the
// packed columns (u_r, u_theta), (u_z, o_r), (o_theta, o_z), (w_r, w_theta),
// (w_z, G_rr), (G_rtheta, G_rz), (G_thetar, G_thetatheta), (G_thetaz, G_zr),
// (G_ztheta, G_zz), o = curl w, G = grad u:
//   P = -u x o - 2 G . w,  (G . w)_i = sum_j G_ij w_j;  out: (P_r, P_theta), (P_z, 0)
template <class T2>
__device__ __forceinline__ void cadj_products(const T2* row, T2* out) {
    using T = typename RealOf<T2>::T;
    const T ur = row[0].x, ut = row[0].y, uz = row[1].x;
    const T orr = row[1].y, ot = row[2].x, oz = row[2].y;
    const T wr = row[3].x, wt = row[3].y, wz = row[4].x;
    const T Grr = row[4].y, Grt = row[5].x, Grz = row[5].y;
    const T Gtr = row[6].x, Gtt = row[6].y, Gtz = row[7].x;
    const T Gzr = row[7].y, Gzt = row[8].x, Gzz = row[8].y;
    const T pr = -(ut * oz - uz * ot) - (T)2 * (Grr * wr + Grt * wt + Grz * wz);
    const T pt = -(uz * orr - ur * oz) - (T)2 * (Gtr * wr + Gtt * wt + Gtz * wz);
    const T pz = -(ur * ot - ut * orr) - (T)2 * (Gzr * wr + Gzt * wt + Gzz * wz);
    out[0] = mk<T2>(pr, pt);
    out[1] = mk<T2>(pz, 0);
}

// ------------------------------------------------------------------ z pass + products
// One block per (j, theta_a) row.  The Hermitian z spectra of two real fields
// are packed into one complex inverse FFT; the pointwise products of the
// physical fields are formed; two real products are packed into one forward
// FFT and separated; the result is truncated to k <= K and scaled.
//   ZFWD: inputs u (3), w (3)          -> outputs u x w (3)
//   ZADJ: inputs u (3), w (3), g (3)   -> outputs w x g (3), g x u (3)
template <class T2, int MODE>
__global__ void k_zpass(Geo g, const T2* __restrict__ Y, T2* __restrict__ Z, ZScales sc, const T2* __restrict__ twg) {
    grid_dep_sync();
    using T = typename RealOf<T2>::T;
    constexpr int NIN = MODE == ZFWD ? 6 : (MODE == ZADJ ? 9 : 18);
    constexpr int NPI = (NIN + 1) / 2;
    constexpr int NOUT = MODE == ZADJ ? 6 : 3;
    constexpr int NPO = (NOUT + 1) / 2;
    constexpr int LD = NPI;  // NPI >= NPO
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = g.nzp, K = g.K, nk = g.nk;
    T2* bufA = reinterpret_cast<T2*>(smem);
    T2* bufB = bufA + N * LD;
    T2* tw = bufB + N * LD;
    const int a = blockIdx.x, j = blockIdx.y;
    const size_t poff = (size_t)g.slot[blockIdx.z] * g.ps;  // batch entry blockIdx.z
    Y += poff;
    Z += poff;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
    // Hermitian-extended spectra, two fields per column
    for (int p = 0; p < NPI; ++p)
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        int k = -1;
        bool neg = false;
        if (n <= K) k = n;
        else if (n >= N - K) { k = N - n; neg = true; }
        T2 q = mk<T2>(0, 0);
        if (k >= 0) {
            const int f1 = 2 * p, f2 = 2 * p + 1;
            T2 y1 = Y[((size_t)(f1 * g.nr + j) * g.nt + a) * nk + k];
            T2 h1 = k == 0 ? mk<T2>(zs<T>(sc.h0, sc.fh0, f1) * y1.x, 0)
                           : mk<T2>(zs<T>(sc.hk, sc.fhk, f1) * y1.x, zs<T>(sc.hk, sc.fhk, f1) * y1.y);
            T2 h2 = mk<T2>(0, 0);
            if (f2 < NIN) {
                T2 y2 = Y[((size_t)(f2 * g.nr + j) * g.nt + a) * nk + k];
                h2 = k == 0 ? mk<T2>(zs<T>(sc.h0, sc.fh0, f2) * y2.x, 0)
                            : mk<T2>(zs<T>(sc.hk, sc.fhk, f2) * y2.x, zs<T>(sc.hk, sc.fhk, f2) * y2.y);
            }
            if (!neg) q = mk<T2>(h1.x - h2.y, h1.y + h2.x);   // H1 + i H2
            else q = mk<T2>(h1.x + h2.y, -h1.y + h2.x);       // conj(H1) + i conj(H2)
        }
        bufA[n * LD + p] = q;
    }
    __syncthreads();
    T2* ph = fft_cols<T2, NPI, LD, +1>(bufA, bufB, N, tw);
    T2* pr = (ph == bufA) ? bufB : bufA;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const T2* row = ph + n * LD;
        const T ur = row[0].x, ut = row[0].y, uz = row[1].x;
        const T wr = row[1].y, wt = row[2].x, wz = row[2].y;
        T2* o = pr + n * LD;
        if (MODE == ZFWD) {
            o[0] = mk<T2>(ut * wz - uz * wt, uz * wr - ur * wz);
            o[1] = mk<T2>(ur * wt - ut * wr, 0);
        } else if (MODE == ZCADJ) {
            cadj_products<T2>(row, o);
        } else {
            const T gr = row[3].x, gt = row[3].y, gz = row[4].x;
            // w x g
            o[0] = mk<T2>(wt * gz - wz * gt, wz * gr - wr * gz);
            // (w x g)_z, (g x u)_r
            o[1] = mk<T2>(wr * gt - wt * gr, gt * uz - gz * ut);
            // (g x u)_theta, (g x u)_z
            o[2] = mk<T2>(gz * ur - gr * uz, gr * ut - gt * ur);
        }
    }
    __syncthreads();
    T2* sp = fft_cols<T2, NPO, LD, -1>(pr, ph, N, tw);
    for (int p = 0; p < NPO; ++p)
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const T2 P = sp[k * LD + p];
        const T2 Pm = sp[((N - k) % N) * LD + p];
        const int o1 = 2 * p, o2 = 2 * p + 1;
        const T s1 = k == 0 ? zs<T>(sc.o0, sc.fo0, o1) : zs<T>(sc.ok, sc.fok, o1);
        T2 z1 = mk<T2>((T)0.5 * (P.x + Pm.x) * s1, (T)0.5 * (P.y - Pm.y) * s1);
        Z[((size_t)(o1 * g.nr + j) * g.nt + a) * nk + k] = z1;
        if (o2 < NOUT) {
            const T s2 = k == 0 ? zs<T>(sc.o0, sc.fo0, o2) : zs<T>(sc.ok, sc.fok, o2);
            T2 z2 = mk<T2>((T)0.5 * (P.y + Pm.y) * s2, (T)-0.5 * (P.x - Pm.x) * s2);
            Z[((size_t)(o2 * g.nr + j) * g.nt + a) * nk + k] = z2;
        }
    }
}

// ------------------------------------------------------------------ theta analysis
// X_f[j][m][k] = sum_a Z_f[j][a][k] e^{-i m theta_a}, |m| <= M, with the k = 0
// plane projected onto Hermitian symmetry.
template <class T2, int KB>
__global__ void k_anal_theta(Geo g, FieldPtrs f, const T2* __restrict__ Z, const T2* __restrict__ twg) {
    grid_dep_sync();
    extern __shared__ __align__(16) unsigned char smem[];
    T2* buf0 = reinterpret_cast<T2*>(smem);
    T2* buf1 = buf0 + g.nt * KB;
    T2* tw = buf1 + g.nt * KB;
    const int k0 = blockIdx.x * KB, j = blockIdx.y;
    const int nf = gridDim.z / g.nb, b = blockIdx.z / nf, fi = blockIdx.z - b * nf, slot = g.slot[b];
    const size_t off = (size_t)slot * g.fs;
    Z += (size_t)slot * g.ps;
    const int kw = min(KB, g.nk - k0);
    for (int i = threadIdx.x; i < g.nt; i += blockDim.x) tw[i] = twg[i];
    const T2* src = Z + ((size_t)(fi * g.nr + j) * g.nt) * g.nk;
    for (int i = threadIdx.x; i < g.nt * KB; i += blockDim.x) {
        const int a = i / KB, kk = i % KB;
        buf0[i] = kk < kw ? src[(size_t)a * g.nk + k0 + kk] : mk<T2>(0, 0);
    }
    __syncthreads();
    T2* res = fft_cols<T2, KB, KB, -1>(buf0, buf1, g.nt, tw);
    const size_t base = off + (size_t)j * g.nm * g.nk;
    float2* dstf = f.outf[fi] ? f.outf[fi] + base : nullptr;
    double2* dst = dstf ? nullptr : f.out[fi] + base;
    const double2* add = f.add[fi] ? f.add[fi] + base : nullptr;
    for (int i = threadIdx.x; i < g.nm * KB; i += blockDim.x) {
        const int im = i / KB, kk = i % KB;
        if (kk >= kw) continue;
        const int m = im - g.M;
        const size_t o = (size_t)im * g.nk + k0 + kk;
        if (dstf) {
            using T = typename RealOf<T2>::T;
            T2 v = res[(m < 0 ? m + g.nt : m) * KB + kk];
            if (k0 + kk == 0) {
                const T2 vm = res[(m > 0 ? g.nt - m : -m) * KB + kk];
                v = mk<T2>((T)0.5 * (v.x + vm.x), (T)0.5 * (v.y - vm.y));
            }
            dstf[o] = to_f(v);
            continue;
        }
        double2 v = to_d(res[(m < 0 ? m + g.nt : m) * KB + kk]);
        if (k0 + kk == 0) {
            double2 vm = to_d(res[(m > 0 ? g.nt - m : -m) * KB + kk]);
            v = make_double2(0.5 * (v.x + vm.x), 0.5 * (v.y - vm.y));
        }
        if (add) v = make_double2(v.x + add[o].x, v.y + add[o].y);
        dst[o] = v;
    }
}

// ------------------------------------------------------------------ two-pass register FFT
// A length N = N1 N2 transform as N2 DFTs of length N1 on stride-N2
// subsequences, a twiddle W_N^{n2 k1}, and N1 DFTs of length N2 on
// contiguous runs (Cooley-Tukey with one shared-memory exchange).  Each DFT
// runs in the registers of one thread, fully unrolled, with its internal
// twiddles folded to compile-time constants.  The inverse transforms below
// take the spectrum in natural order and leave physical index k1 + N1 k2 in
// slot k2 + N2 k1; the forward transforms take that slot order back to a
// natural-order spectrum.  The physical-space work in between is pointwise,
// so the permutation never has to be undone.

// cos and sin of 2 pi e / L evaluated by the compiler: e is reduced to a
// quadrant with integer arithmetic, the remaining angle x in [0, pi/2) goes
// through the Taylor series of sin and cos (16 terms, below 1e-17 there).
namespace ct {
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr double tsin(double x) {
    double t = x, s = x;
    for (int i = 1; i < 16; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double tcos(double x) {
    double t = 1.0, s = 1.0;
    for (int i = 1; i < 16; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double cos2pi(long e, long L) {
    const long n = ((e % L) + L) % L, q = 4 * n / L;
    const double x = kTwoPi * (double)(4 * n - q * L) / (4.0 * (double)L);
    return q == 0 ? tcos(x) : q == 1 ? -tsin(x) : q == 2 ? -tcos(x) : tsin(x);
}
__host__ __device__ constexpr double sin2pi(long e, long L) {
    const long n = ((e % L) + L) % L, q = 4 * n / L;
    const double x = kTwoPi * (double)(4 * n - q * L) / (4.0 * (double)L);
    return q == 0 ? tsin(x) : q == 1 ? tcos(x) : q == 2 ? -tsin(x) : -tcos(x);
}
}  // namespace ct

// x e^{SIGN 2 pi i E / L} for a compile-time exponent E
template <class T2, int L, int SIGN, int E>
__device__ __forceinline__ T2 twc(T2 x) {
    using T = typename RealOf<T2>::T;
    constexpr int e = ((E % L) + L) % L;
    if constexpr (e == 0) {
        return x;
    } else if constexpr (2 * e == L) {
        return mk<T2>(-x.x, -x.y);
    } else if constexpr (4 * e == L) {  // SIGN i
        return SIGN > 0 ? mk<T2>(-x.y, x.x) : mk<T2>(x.y, -x.x);
    } else if constexpr (4 * e == 3 * L) {  // -SIGN i
        return SIGN > 0 ? mk<T2>(x.y, -x.x) : mk<T2>(-x.y, x.x);
    } else {
        constexpr T c = (T)ct::cos2pi(e, L);
        constexpr T sn = (T)(SIGN * ct::sin2pi(e, L));
        return mk<T2>(c * x.x - sn * x.y, c * x.y + sn * x.x);
    }
}

// x e^{SIGN 2 pi i e / N} for a run-time exponent 0 <= e < N, from the table
// tw[n] = e^{-2 pi i n / N}
template <class T2, int SIGN>
__device__ __forceinline__ T2 twr(T2 x, const T2* tw, int e) {
    T2 w = tw[e];
    if (SIGN > 0) w.y = -w.y;
    return cmul(x, w);
}

template <class T2, int L, int SIGN, int R, int Q, int... I>
__device__ __forceinline__ void rtwiddle(T2 (&s)[R][Q], std::integer_sequence<int, I...>) {
    ((s[I / Q][I % Q] = twc<T2, L, SIGN, (I / Q) * (I % Q)>(s[I / Q][I % Q])), ...);
}

// In-register DFT X[k] = sum_n v[n] e^{SIGN 2 pi i n k / L}, L = 2^a 3^b:
// radix-2/3/4 butterflies at the leaves, mixed-radix Cooley-Tukey above them
// (n = a + R b, k = kb + Q ka).
template <class T2, int L, int SIGN>
__device__ __forceinline__ void rdft(T2 (&v)[L]) {
    using T = typename RealOf<T2>::T;
    if constexpr (L == 1) {
    } else if constexpr (L == 2) {
        const T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (L == 3) {
        constexpr T h = (T)(SIGN * 0.86602540378443864676);  // SIGN sqrt(3)/2
        const T2 t1 = cadd(v[1], v[2]);
        const T2 t2 = mk<T2>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        const T2 t3 = imul(csub(v[1], v[2]), h);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if constexpr (L == 4) {
        const T2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const T2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        const T2 id = imul(d13, (T)SIGN);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, id);
        v[3] = csub(d02, id);
    } else {
        constexpr int R = (L % 4 == 0) ? 4 : ((L % 2 == 0) ? 2 : 3);
        constexpr int Q = L / R;
        T2 s[R][Q];
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < Q; ++b) s[a][b] = v[a + R * b];
#pragma unroll
        for (int a = 0; a < R; ++a) rdft<T2, Q, SIGN>(s[a]);
        rtwiddle<T2, L, SIGN, R, Q>(s, std::make_integer_sequence<int, R * Q>{});
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            T2 t[R];
#pragma unroll
            for (int a = 0; a < R; ++a) t[a] = s[a][b];
            rdft<T2, R, SIGN>(t);
#pragma unroll
            for (int a = 0; a < R; ++a) v[b + Q * a] = t[a];
        }
    }
}

// theta synthesis, two-pass: block (k tile of KB, j, field) of kT2 threads,
// KB * N1 or KB * N2 tasks per pass.  Slot s of the output rows holds theta
// index (s / N2) + N1 (s % N2).  The task counts are multiples of the block
// size, so each thread runs a fixed number of tasks; in FP32, where their
// inputs fit in registers (at most 24 values), it loads all of them before the
// first DFT, so that one memory latency is exposed per pass instead of one per
// task, and runs at 64 registers (eight blocks per SM).
constexpr int kT2 = 128;
template <class T2, int KB, int N1, int N2>
__global__ void __launch_bounds__(kT2, sizeof(T2) == 8 ? 8 : 1)
    k_synth2(Geo g, FieldPtrs f, T2* __restrict__ Y, const T2* __restrict__ twg) {
    grid_dep_sync();
    constexpr int N = N1 * N2, IT1 = KB * N2 / kT2, IT2 = KB * N1 / kT2;
    static_assert(KB * N2 % kT2 == 0 && KB * N1 % kT2 == 0, "whole tasks per thread");
    extern __shared__ __align__(16) unsigned char smem[];
    T2* buf = reinterpret_cast<T2*>(smem);  // [N][KB]
    T2* tw = buf + N * KB;                   // [N]
    const int k0 = blockIdx.x * KB, j = blockIdx.y;
    const int nf = gridDim.z / g.nb, b = blockIdx.z / nf, fi = blockIdx.z - b * nf, slot = g.slot[b];
    Y += (size_t)slot * g.ps;
    for (int i = threadIdx.x; i < N; i += kT2) tw[i] = twg[i];
    const size_t base = (size_t)slot * g.fs + (size_t)j * g.nm * g.nk;
    const float2* srcf = f.inf[fi] ? f.inf[fi] + base : nullptr;
    const double2* src = srcf ? nullptr : f.in[fi] + base;
    auto load = [&](int it, T2 (&v)[N1]) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, n2 = t / KB, k = k0 + kk;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int n = n2 + N2 * n1;  // m mod N; zero padding for |m| > M
            const int m = n <= g.M ? n : n - N;
            v[n1] = (k < g.nk && m >= -g.M) ? synth_in<T2>(src, srcf, (size_t)(m + g.M) * g.nk + k) : mk<T2>(0, 0);
        }
    };
    auto dft1 = [&](int it, T2 (&v)[N1]) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, n2 = t / KB;
        rdft<T2, N1, +1>(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[(n2 + N2 * k1) * KB + kk] = twr<T2, +1>(v[k1], tw, n2 * k1);
    };
    if constexpr (sizeof(T2) == 8 && IT1 * N1 <= 24) {  // FP32 values only: FP64 ones would spill
        T2 v[IT1][N1];
#pragma unroll
        for (int it = 0; it < IT1; ++it) load(it, v[it]);
        __syncthreads();  // twiddles
#pragma unroll
        for (int it = 0; it < IT1; ++it) dft1(it, v[it]);
    } else {
        __syncthreads();  // twiddles
#pragma unroll 1
        for (int it = 0; it < IT1; ++it) {
            T2 v[N1];
            load(it, v);
            dft1(it, v);
        }
    }
    __syncthreads();
    T2* dst = Y + ((size_t)(fi * g.nr + j) * N) * g.nk;
    constexpr int kUnroll2 = sizeof(T2) == 8 ? IT2 : 1;  // FP64 tasks one at a time (registers)
#pragma unroll kUnroll2
    for (int it = 0; it < IT2; ++it) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, k1 = t / KB, k = k0 + kk;
        T2 v[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v[n2] = buf[(N2 * k1 + n2) * KB + kk];
        rdft<T2, N2, +1>(v);
        if (k < g.nk) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) dst[(size_t)(N2 * k1 + k2) * g.nk + k] = v[k2];
        }
    }
}

// theta analysis, two-pass (input rows in the slot order of k_synth2), with
// the k = 0 plane projected onto Hermitian symmetry.  Same thread layout as
// k_synth2; the first pass loads all its inputs before its DFTs where they
// fit in registers, and each task of the second pass loads the values to add
// (the base-flow terms) before its DFT.
template <class T2, int KB, int N1, int N2>
__global__ void __launch_bounds__(kT2, sizeof(T2) == 8 ? 6 : 1) k_anal2(Geo g, FieldPtrs f, const T2* __restrict__ Z,
                                               const T2* __restrict__ twg) {
    grid_dep_sync();
    constexpr int N = N1 * N2, IT1 = KB * N1 / kT2, IT2 = KB * N2 / kT2;
    static_assert(KB * N2 % kT2 == 0 && KB * N1 % kT2 == 0, "whole tasks per thread");
    extern __shared__ __align__(16) unsigned char smem[];
    T2* buf = reinterpret_cast<T2*>(smem);  // [N][KB]
    T2* tw = buf + N * KB;                   // [N]
    const int k0 = blockIdx.x * KB, j = blockIdx.y;
    const int nf = gridDim.z / g.nb, b = blockIdx.z / nf, fi = blockIdx.z - b * nf, slot = g.slot[b];
    const size_t off = (size_t)slot * g.fs;
    Z += (size_t)slot * g.ps;
    for (int i = threadIdx.x; i < N; i += kT2) tw[i] = twg[i];
    const T2* src = Z + ((size_t)(fi * g.nr + j) * N) * g.nk;
    auto load = [&](int it, T2 (&v)[N2]) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, k1 = t / KB, k = k0 + kk;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v[n2] = k < g.nk ? src[(size_t)(N2 * k1 + n2) * g.nk + k] : mk<T2>(0, 0);
    };
    auto dft1 = [&](int it, T2 (&v)[N2]) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, k1 = t / KB;
        rdft<T2, N2, -1>(v);
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) buf[(N2 * k1 + m2) * KB + kk] = twr<T2, -1>(v[m2], tw, k1 * m2);
    };
    if constexpr (sizeof(T2) == 8 && IT1 * N2 <= 24) {  // FP32 values only: FP64 ones would spill
        T2 v[IT1][N2];
#pragma unroll
        for (int it = 0; it < IT1; ++it) load(it, v[it]);
        __syncthreads();  // twiddles
#pragma unroll
        for (int it = 0; it < IT1; ++it) dft1(it, v[it]);
    } else {
        __syncthreads();  // twiddles
#pragma unroll 1
        for (int it = 0; it < IT1; ++it) {
            T2 v[N2];
            load(it, v);
            dft1(it, v);
        }
    }
    __syncthreads();
    const size_t base = off + (size_t)j * g.nm * g.nk;
    float2* dstf = f.outf[fi] ? f.outf[fi] + base : nullptr;
    double2* dst = dstf ? nullptr : f.out[fi] + base;
    const double2* add = f.add[fi] ? f.add[fi] + base : nullptr;
#pragma unroll 1
    for (int it = 0; it < IT2; ++it) {
        const int t = threadIdx.x + it * kT2, kk = t % KB, m2 = t / KB, k = k0 + kk;
        constexpr bool kEarly = sizeof(T2) == 8 && N1 <= 8;  // larger or FP64 tasks: no room in registers
        double2 ad[kEarly ? N1 : 1];
        if constexpr (kEarly) {
#pragma unroll
            for (int m1 = 0; m1 < N1; ++m1) {
                const int n = m2 + N2 * m1;
                const int m = n <= g.M ? n : n - N;
                ad[m1] = (add && k > 0 && k < g.nk && m >= -g.M) ? add[(size_t)(m + g.M) * g.nk + k]
                                                                  : make_double2(0, 0);
            }
        }
        T2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = buf[(m2 + N2 * k1) * KB + kk];
        rdft<T2, N1, -1>(v);
#pragma unroll
        for (int m1 = 0; m1 < N1; ++m1) {
            const int n = m2 + N2 * m1;
            const int m = n <= g.M ? n : n - N;
            if (k < g.nk && m >= -g.M) {
                if (k == 0) {
                    buf[n * KB + kk] = v[m1];
                } else if (dstf) {
                    dstf[(size_t)(m + g.M) * g.nk + k] = to_f(v[m1]);
                } else {
                    const size_t o = (size_t)(m + g.M) * g.nk + k;
                    double2 x = to_d(v[m1]);
                    if (add) {
                        const double2 a = kEarly ? ad[kEarly ? m1 : 0] : add[o];
                        x = make_double2(x.x + a.x, x.y + a.y);
                    }
                    dst[o] = x;
                }
            }
        }
    }
    if (k0 == 0) {  // block-uniform
        __syncthreads();
        for (int im = threadIdx.x; im < g.nm; im += blockDim.x) {
            const int m = im - g.M;
            if (dstf) {
                using T = typename RealOf<T2>::T;
                const T2 v = buf[(m < 0 ? m + N : m) * KB], vm = buf[(m > 0 ? N - m : -m) * KB];
                dstf[(size_t)im * g.nk] = to_f(mk<T2>((T)0.5 * (v.x + vm.x), (T)0.5 * (v.y - vm.y)));
                continue;
            }
            const double2 v = to_d(buf[(m < 0 ? m + N : m) * KB]);
            const double2 vm = to_d(buf[(m > 0 ? N - m : -m) * KB]);
            double2 x = make_double2(0.5 * (v.x + vm.x), 0.5 * (v.y - vm.y));
            if (add) x = make_double2(x.x + add[(size_t)im * g.nk].x, x.y + add[(size_t)im * g.nk].y);
            dst[(size_t)im * g.nk] = x;
        }
    }
}

// Compile-time loop: f(std::integral_constant<int, 0>()) ... f(<N - 1>).
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>()), ...);
}
template <int N, class F> __device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>());
}

// z pass, two-pass FFTs in place in padded shared-memory columns (one gap
// after every run of N2 slots keeps both access patterns free of bank
// conflicts), RB rows (theta indices a) of one radial index per block.  The
// spectra are 3/2-padded: K = N/3 - 1 is a compile-time constant here (the
// launcher checks it), so the inverse pass knows at compile time which of its
// strided inputs fall in the zero band K < n < N - K and loads none of them,
// and the forward pass stores no output of that band (the separation never
// reads it).  Same contract as k_zpass.
template <class T2, int MODE, int N1, int N2, int RB>
__global__ void __launch_bounds__(96, 6)
    k_zpass2(Geo g, const T2* __restrict__ Y, T2* __restrict__ Z, ZScales sc, const T2* __restrict__ twg) {
    grid_dep_sync();
    using T = typename RealOf<T2>::T;
    constexpr int N = N1 * N2, NP = N + N1, KC = N / 3 - 1, NK = KC + 1;
    constexpr int NIN = MODE == ZFWD ? 6 : (MODE == ZADJ ? 9 : 18);
    constexpr int NPI = (NIN + 1) / 2;
    constexpr int NOUT = MODE == ZADJ ? 6 : 3;
    constexpr int NPO = (NOUT + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    T2* col = reinterpret_cast<T2*>(smem);  // [RB][NPI][NP]
    T2* tw = col + RB * NPI * NP;            // [N]
    const int a0 = blockIdx.x * RB, j = blockIdx.y;
    const size_t poff = (size_t)g.slot[blockIdx.z] * g.ps;  // batch entry blockIdx.z
    Y += poff;
    Z += poff;
    auto at = [](int s) { return s + s / N2; };
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    // inverse, strided pass: Hermitian-extended spectra, two real fields per column
    for (int t = threadIdx.x; t < RB * NPI * N2; t += blockDim.x) {
        const int r = t / (NPI * N2), pn = t - r * (NPI * N2), p = pn / N2, n2 = pn - p * N2;
        const int f1 = 2 * p, f2 = 2 * p + 1;
        const bool has2 = f2 < NIN;
        const T2* y1 = Y + ((size_t)(f1 * g.nr + j) * g.nt + a0 + r) * NK;
        const T2* y2 = Y + ((size_t)((has2 ? f2 : f1) * g.nr + j) * g.nt + a0 + r) * NK;
        const T h01 = zs<T>(sc.h0, sc.fh0, f1), hk1 = zs<T>(sc.hk, sc.fhk, f1);
        const T h02 = has2 ? zs<T>(sc.h0, sc.fh0, f2) : (T)0, hk2 = has2 ? zs<T>(sc.hk, sc.fhk, f2) : (T)0;
        // H1 + i H2 at z-wavenumber k (positive side) or conj(H1) + i conj(H2)
        // (negative side); only k = 0 drops its imaginary parts
        auto entry = [&](int k, bool neg, bool may0) {
            const T2 a1 = y1[k], a2 = has2 ? y2[k] : mk<T2>(0, 0);
            const bool z0 = may0 && k == 0;
            const T2 h1 = z0 ? mk<T2>(h01 * a1.x, 0) : mk<T2>(hk1 * a1.x, hk1 * a1.y);
            const T2 h2 = z0 ? mk<T2>(h02 * a2.x, 0) : mk<T2>(hk2 * a2.x, hk2 * a2.y);
            return !neg ? mk<T2>(h1.x - h2.y, h1.y + h2.x) : mk<T2>(h1.x + h2.y, -h1.y + h2.x);
        };
        T2 v[N1];
        static_for<N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            constexpr int lo = N2 * n1, hi = lo + N2 - 1;
            const int n = n2 + lo;
            if constexpr (hi <= KC) {
                v[n1] = entry(n, false, n1 == 0);
            } else if constexpr (lo >= N - KC) {
                v[n1] = entry(N - n, true, false);
            } else if constexpr (lo > KC && hi < N - KC) {
                v[n1] = mk<T2>(0, 0);
            } else {
                v[n1] = n <= KC ? entry(n, false, n1 == 0) : (n >= N - KC ? entry(N - n, true, false) : mk<T2>(0, 0));
            }
        });
        rdft<T2, N1, +1>(v);
        T2* c = col + (r * NPI + p) * NP;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) c[at(n2 + N2 * k1)] = twr<T2, +1>(v[k1], tw, n2 * k1);
    }
    __syncthreads();
    // inverse, contiguous pass: physical values
    for (int t = threadIdx.x; t < RB * NPI * N1; t += blockDim.x) {
        const int rp = t / N1, k1 = t - rp * N1;
        T2* c = col + rp * NP;
        T2 v[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) v[n2] = c[at(N2 * k1 + n2)];
        rdft<T2, N2, +1>(v);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) c[at(N2 * k1 + k2)] = v[k2];
    }
    __syncthreads();
    // pointwise products, in place (each slot read and written by one thread)
    for (int t = threadIdx.x; t < RB * N; t += blockDim.x) {
        const int r = t / N, s = t - r * N;
        T2* c = col + r * NPI * NP;
        const int o = at(s);
        if constexpr (MODE == ZCADJ) {
            T2 row[NPI], res[2];
#pragma unroll
            for (int p = 0; p < NPI; ++p) row[p] = c[p * NP + o];
            cadj_products<T2>(row, res);
            c[o] = res[0];
            c[NP + o] = res[1];
            continue;
        }
        const T2 c0 = c[o], c1 = c[NP + o], c2 = c[2 * NP + o];
        const T ur = c0.x, ut = c0.y, uz = c1.x;
        const T wr = c1.y, wt = c2.x, wz = c2.y;
        if (MODE == ZFWD) {
            c[o] = mk<T2>(ut * wz - uz * wt, uz * wr - ur * wz);
            c[NP + o] = mk<T2>(ur * wt - ut * wr, 0);
        } else {
            const T2 c3 = c[3 * NP + o], c4 = c[4 * NP + o];
            const T gr = c3.x, gt = c3.y, gz = c4.x;
            c[o] = mk<T2>(wt * gz - wz * gt, wz * gr - wr * gz);           // w x g
            c[NP + o] = mk<T2>(wr * gt - wt * gr, gt * uz - gz * ut);      // (w x g)_z, (g x u)_r
            c[2 * NP + o] = mk<T2>(gz * ur - gr * uz, gr * ut - gt * ur);  // (g x u)_theta, (g x u)_z
        }
    }
    __syncthreads();
    // forward, contiguous pass
    for (int t = threadIdx.x; t < RB * NPO * N1; t += blockDim.x) {
        const int r = t / (NPO * N1), pk = t - r * (NPO * N1), p = pk / N1, k1 = pk - p * N1;
        T2* c = col + (r * NPI + p) * NP;
        T2 v[N2];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = c[at(N2 * k1 + k2)];
        rdft<T2, N2, -1>(v);
#pragma unroll
        for (int m2 = 0; m2 < N2; ++m2) c[at(N2 * k1 + m2)] = twr<T2, -1>(v[m2], tw, k1 * m2);
    }
    __syncthreads();
    // forward, strided pass: natural-order spectra, the zero band left out
    for (int t = threadIdx.x; t < RB * NPO * N2; t += blockDim.x) {
        const int r = t / (NPO * N2), pm = t - r * (NPO * N2), p = pm / N2, m2 = pm - p * N2;
        T2* c = col + (r * NPI + p) * NP;
        T2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = c[at(m2 + N2 * k1)];
        rdft<T2, N1, -1>(v);
        static_for<N1>([&](auto I) {
            constexpr int m1 = decltype(I)::value;
            constexpr int lo = N2 * m1, hi = lo + N2 - 1;
            if constexpr (!(lo > KC && hi < N - KC)) c[at(m2 + lo)] = v[m1];
        });
    }
    __syncthreads();
    // separate the two real products of each column, truncate to k <= K, scale
    for (int t = threadIdx.x; t < RB * NPO * NK; t += blockDim.x) {
        const int r = t / (NPO * NK), pk = t - r * (NPO * NK), p = pk / NK, k = pk - p * NK;
        const T2* c = col + (r * NPI + p) * NP;
        const T2 P = c[at(k)];
        const T2 Pm = c[at((N - k) % N)];
        const int o1 = 2 * p, o2 = 2 * p + 1;
        const size_t row = (size_t)j * g.nt + a0 + r;
        const T s1 = k == 0 ? zs<T>(sc.o0, sc.fo0, o1) : zs<T>(sc.ok, sc.fok, o1);
        Z[((size_t)o1 * g.nr * g.nt + row) * NK + k] = mk<T2>((T)0.5 * (P.x + Pm.x) * s1, (T)0.5 * (P.y - Pm.y) * s1);
        if (o2 < NOUT) {
            const T s2 = k == 0 ? zs<T>(sc.o0, sc.fo0, o2) : zs<T>(sc.ok, sc.fok, o2);
            Z[((size_t)o2 * g.nr * g.nt + row) * NK + k] =
                mk<T2>((T)0.5 * (P.y + Pm.y) * s2, (T)-0.5 * (P.x - Pm.x) * s2);
        }
    }
}

// ------------------------------------------------------------------ launchers
template <class T2> static const T2* tw_theta(const Twiddles& t);
template <> const double2* tw_theta<double2>(const Twiddles& t) { return t.th_d; }
template <> const float2* tw_theta<float2>(const Twiddles& t) { return t.th_f; }
template <class T2> static const T2* tw_z(const Twiddles& t);
template <> const double2* tw_z<double2>(const Twiddles& t) { return t.z_d; }
template <> const float2* tw_z<float2>(const Twiddles& t) { return t.z_f; }

template <class T2> static int theta_kb(const Geo& g) {
    int kb = 32;
    while (kb > 4 && (kb / 2 >= g.nk || (size_t)(2 * g.nt * kb + g.nt) * sizeof(T2) > 100 * 1024)) kb /= 2;
    return kb;
}

template <class T2, int KB>
static void synth_theta_kb(const Geo& g, const FieldPtrs& f, int nfield, T2* Y, const T2* tw, cudaStream_t s) {
    const size_t sm = (size_t)(2 * g.nt * KB + g.nt) * sizeof(T2);
    smem_limit((const void*)k_synth_theta<T2, KB>);
    dim3 grid((g.nk + KB - 1) / KB, g.nr, nfield * g.nb);
    launch_pdl(k_synth_theta<T2, KB>, grid, 256, sm, s, g, f, Y, tw);
}

template <class T2, int KB>
static void anal_theta_kb(const Geo& g, const FieldPtrs& f, int nfield, const T2* Z, const T2* tw, cudaStream_t s) {
    const size_t sm = (size_t)(2 * g.nt * KB + g.nt) * sizeof(T2);
    smem_limit((const void*)k_anal_theta<T2, KB>);
    dim3 grid((g.nk + KB - 1) / KB, g.nr, nfield * g.nb);
    launch_pdl(k_anal_theta<T2, KB>, grid, 256, sm, s, g, f, Z, tw);
}

// Two-pass register kernels serve the lengths with a split N = N1 N2 below;
// the Stockham kernels serve every other 2^a 3^b length.  The theta kernels
// take KB k-columns per block.
template <class T2, int KB, int N1, int N2>
static void synth2(const Geo& g, const FieldPtrs& f, int nfield, T2* Y, const T2* tw, cudaStream_t s) {
    const size_t sm = (size_t)(N1 * N2 * KB + N1 * N2) * sizeof(T2);
    smem_limit((const void*)k_synth2<T2, KB, N1, N2>);
    dim3 grid((g.nk + KB - 1) / KB, g.nr, nfield * g.nb);
    launch_pdl(k_synth2<T2, KB, N1, N2>, grid, kT2, sm, s, g, f, Y, tw);
}
template <class T2, int KB, int N1, int N2>
static void anal2(const Geo& g, const FieldPtrs& f, int nfield, const T2* Z, const T2* tw, cudaStream_t s) {
    const size_t sm = (size_t)(N1 * N2 * KB + N1 * N2) * sizeof(T2);
    smem_limit((const void*)k_anal2<T2, KB, N1, N2>);
    dim3 grid((g.nk + KB - 1) / KB, g.nr, nfield * g.nb);
    launch_pdl(k_anal2<T2, KB, N1, N2>, grid, kT2, sm, s, g, f, Z, tw);
}

template <class T2>
void launch_synth_theta(const Geo& g, const FieldPtrs& f, int nfield, T2* Y, const Twiddles& tw, cudaStream_t s) {
    switch (g.nt) {
        case 96: synth2<T2, 32, 8, 12>(g, f, nfield, Y, tw_theta<T2>(tw), s); check_launch("synth_theta"); return;
        case 192: synth2<T2, 32, 16, 12>(g, f, nfield, Y, tw_theta<T2>(tw), s); check_launch("synth_theta"); return;
        case 384: synth2<T2, 16, 16, 24>(g, f, nfield, Y, tw_theta<T2>(tw), s); check_launch("synth_theta"); return;
        default: break;
    }
    switch (theta_kb<T2>(g)) {
        case 32: synth_theta_kb<T2, 32>(g, f, nfield, Y, tw_theta<T2>(tw), s); break;
        case 16: synth_theta_kb<T2, 16>(g, f, nfield, Y, tw_theta<T2>(tw), s); break;
        case 8: synth_theta_kb<T2, 8>(g, f, nfield, Y, tw_theta<T2>(tw), s); break;
        default: synth_theta_kb<T2, 4>(g, f, nfield, Y, tw_theta<T2>(tw), s); break;
    }
    check_launch("synth_theta");
}

template <class T2>
void launch_anal_theta(const Geo& g, const FieldPtrs& f, int nfield, const T2* Z, const Twiddles& tw, cudaStream_t s) {
    switch (g.nt) {
        case 96: anal2<T2, 32, 8, 12>(g, f, nfield, Z, tw_theta<T2>(tw), s); check_launch("anal_theta"); return;
        case 192: anal2<T2, 32, 16, 12>(g, f, nfield, Z, tw_theta<T2>(tw), s); check_launch("anal_theta"); return;
        case 384: anal2<T2, 16, 16, 24>(g, f, nfield, Z, tw_theta<T2>(tw), s); check_launch("anal_theta"); return;
        default: break;
    }
    switch (theta_kb<T2>(g)) {
        case 32: anal_theta_kb<T2, 32>(g, f, nfield, Z, tw_theta<T2>(tw), s); break;
        case 16: anal_theta_kb<T2, 16>(g, f, nfield, Z, tw_theta<T2>(tw), s); break;
        case 8: anal_theta_kb<T2, 8>(g, f, nfield, Z, tw_theta<T2>(tw), s); break;
        default: anal_theta_kb<T2, 4>(g, f, nfield, Z, tw_theta<T2>(tw), s); break;
    }
    check_launch("anal_theta");
}

// N/4 threads divide the radix-4 (and the radix-2, radix-3) stages of a
// length-N column exactly; at least one warp, at most 256.
static unsigned zpass_threads(const Geo& g) {
    const int t = (g.nzp / 4 + 31) / 32 * 32;
    return (unsigned)std::max(32, std::min(256, t));
}

// rows per block of the two-pass z kernel: two for the forward pass (its
// three packed columns then fill the block's threads better, at 22 KB of
// shared memory: 16.6 against 18.4 ms per 64x64x256 gradient), one for the
// adjoint passes, whose five and nine columns fill them already (two rows
// measured slower there: 13.6 against 12.8 ms)
template <int MODE> constexpr int zpass_rows() { return MODE == ZFWD ? 2 : 1; }

template <class T2, int MODE, int N1, int N2, int RB>
static void zpass2(const Geo& g, const T2* Y, T2* Z, const ZScales& sc, const T2* tw, cudaStream_t s) {
    constexpr int NPI = MODE == ZFWD ? 3 : (MODE == ZADJ ? 5 : 9);
    const size_t sm = (size_t)(RB * NPI * (N1 * N2 + N1) + N1 * N2) * sizeof(T2);
    smem_limit((const void*)k_zpass2<T2, MODE, N1, N2, RB>);
    launch_pdl(k_zpass2<T2, MODE, N1, N2, RB>, dim3(g.nt / RB, g.nr, g.nb), zpass_threads(g), sm, s, g, Y, Z, sc,
               tw);
}
template <class T2, int MODE, int N1, int N2>
static void zpass2_rows(const Geo& g, const T2* Y, T2* Z, const ZScales& sc, const T2* tw, cudaStream_t s) {
    constexpr int RB = zpass_rows<MODE>();
    if (g.nt % RB == 0) zpass2<T2, MODE, N1, N2, RB>(g, Y, Z, sc, tw, s);
    else zpass2<T2, MODE, N1, N2, 1>(g, Y, Z, sc, tw, s);
}
// The two-pass kernel serves the 3/2-padded lengths N = 3 (K + 1) below; any
// other length goes to the Stockham kernel.
template <class T2, int MODE>
static bool zpass2_any(const Geo& g, const T2* Y, T2* Z, const ZScales& sc, const T2* tw, cudaStream_t s) {
    if (g.nzp != 3 * g.nk || g.K != g.nk - 1) return false;
    switch (g.nzp) {
        case 96: zpass2_rows<T2, MODE, 8, 12>(g, Y, Z, sc, tw, s); return true;
        case 192: zpass2_rows<T2, MODE, 16, 12>(g, Y, Z, sc, tw, s); return true;
        case 384: zpass2_rows<T2, MODE, 16, 24>(g, Y, Z, sc, tw, s); return true;
        default: return false;
    }
}

template <class T2, int MODE>
static void zpass_stockham(const Geo& g, const T2* Y, T2* Z, const ZScales& sc, const T2* tw, cudaStream_t s) {
    constexpr int LD = MODE == ZFWD ? 3 : (MODE == ZADJ ? 5 : 9);
    const size_t sm = (size_t)(2 * g.nzp * LD + g.nzp) * sizeof(T2);
    smem_limit((const void*)k_zpass<T2, MODE>);
    launch_pdl(k_zpass<T2, MODE>, dim3(g.nt, g.nr, g.nb), zpass_threads(g), sm, s, g, Y, Z, sc, tw);
}

template <class T2>
void launch_zpass(const Geo& g, int mode, const T2* Y, T2* Z, const ZScales& sc_in, const Twiddles& tw, cudaStream_t s) {
    ZScales sc = sc_in;
    for (int i = 0; i < kMaxIn; ++i) {
        sc.fh0[i] = (float)sc.h0[i];
        sc.fhk[i] = (float)sc.hk[i];
    }
    for (int i = 0; i < 6; ++i) {
        sc.fo0[i] = (float)sc.o0[i];
        sc.fok[i] = (float)sc.ok[i];
    }
    const T2* t = tw_z<T2>(tw);
    // FP64 z passes stay on the Stockham kernel: they are bound by the FP64
    // pipe, where the register kernel's lower occupancy measured slower.
    bool done = false;
    if constexpr (std::is_same<T2, float2>::value)
        done = mode == ZFWD ? zpass2_any<T2, ZFWD>(g, Y, Z, sc, t, s)
                            : (mode == ZADJ ? zpass2_any<T2, ZADJ>(g, Y, Z, sc, t, s)
                                            : zpass2_any<T2, ZCADJ>(g, Y, Z, sc, t, s));
    if (!done) {
        if (mode == ZFWD) zpass_stockham<T2, ZFWD>(g, Y, Z, sc, t, s);
        else if (mode == ZADJ) zpass_stockham<T2, ZADJ>(g, Y, Z, sc, t, s);
        else zpass_stockham<T2, ZCADJ>(g, Y, Z, sc, t, s);
    }
    check_launch("zpass");
}

template void launch_synth_theta<double2>(const Geo&, const FieldPtrs&, int, double2*, const Twiddles&, cudaStream_t);
template void launch_synth_theta<float2>(const Geo&, const FieldPtrs&, int, float2*, const Twiddles&, cudaStream_t);
template void launch_anal_theta<double2>(const Geo&, const FieldPtrs&, int, const double2*, const Twiddles&,
                                         cudaStream_t);
template void launch_anal_theta<float2>(const Geo&, const FieldPtrs&, int, const float2*, const Twiddles&,
                                        cudaStream_t);
template void launch_zpass<double2>(const Geo&, int, const double2*, double2*, const ZScales&, const Twiddles&,
                                    cudaStream_t);
template void launch_zpass<float2>(const Geo&, int, const float2*, float2*, const ZScales&, const Twiddles&,
                                   cudaStream_t);

}  // namespace pnop
