// Device kernels of the pseudo-spectral pipe-flow step (Keuchel & Avila,
// Section 2.4) and of its exact discrete transpose (the adjoint step that
// replaces Eq. 2.9-2.11).
//
// Spectral fields are FP64 complex, layout [c][j][m + M][k].  Everything here
// is FP64: the curl and base-flow terms, and everything radial (banded
// matvecs, banded LU solves, influence and flux corrections).  The theta/z
// transforms are in transforms.cu.  Every kernel also serves batched launches:
// it finds its batch entry in one grid dimension and offsets its field
// pointers and per-request tables by that entry's slot (see Geo).
#include "dev_common.cuh"
#include "dev_df.cuh"
#include "kernels.hpp"

#include <algorithm>
#include <string>

namespace pnop {

// ------------------------------------------------------------------ spectral FP64 kernels
struct Idx {
    int j, im, k, m, b, slot;
    size_t S, off;  // off: element offset of the entry's slot in every spectral buffer
};
// Spectral kernels run on a 3-D grid: x covers k, y the azimuthal index, z
// the radial index and the batch entry (z = b nr + j), so no thread divides
// to find its (j, m, k).
__device__ __forceinline__ bool decode(const Geo& g, Idx& d) {
    d.S = (size_t)g.nr * g.nm * g.nk;
    d.k = blockIdx.x * blockDim.x + threadIdx.x;
    d.im = blockIdx.y;
    d.b = blockIdx.z / g.nr;
    d.j = blockIdx.z - d.b * g.nr;
    d.slot = g.slot[d.b];
    d.off = (size_t)d.slot * g.fs;
    d.m = d.im - g.M;
    return d.k < g.nk;
}
// Per-slot operator tables of a batched context (stride 0 tables are shared).
__device__ __forceinline__ const double* slot_Lb(const Geo& g, int slot) { return g.Lb + (size_t)slot * g.sLb; }
__device__ __forceinline__ const double* slot_dgt(const Geo& g, int slot) { return g.dgt + (size_t)slot * g.sNk; }
__device__ __forceinline__ const double* slot_infl(const Geo& g, int slot) { return g.infl + (size_t)slot * g.sInfl; }
__device__ __forceinline__ const double* slot_fluxg(const Geo& g, int slot) { return g.fluxg + (size_t)slot * g.sNr; }
template <class P> __device__ __forceinline__ P moved(P p, size_t off) { return p ? p + off : p; }
__device__ __forceinline__ size_t sidx(const Geo& g, int j, int im, int k) {
    return ((size_t)j * g.nm + im) * g.nk + k;
}

// Banded row product sum_s B[j][s] x[j-4+s].  Every row has at most 9
// nonzeros: columns 0..8 for the one-sided wall rows j < 4, columns j-4..j+4
// (clipped at the axis, where mirrored nodes fold inwards) otherwise.
__device__ __forceinline__ double2 band_row(const Geo& g, const double* B, const double2* x, int j, int im, int k) {
    double2 acc = make_double2(0, 0);
    if (j >= 4) {
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            const int c = j - 4 + s;
            if (c < g.nr) acc = dfma(__ldg(B + s), x[sidx(g, c, im, k)], acc);
        }
    } else {
#pragma unroll
        for (int s = 0; s < kB; ++s) {
            const int c = j - 4 + s;
            if (c >= 0 && c <= 8) acc = dfma(__ldg(B + s), x[sidx(g, c, im, k)], acc);
        }
    }
    return acc;
}
// Transposed banded product (B^T x)_j = sum_{j'} B[j'][j - j' + 4] x[j'].
// Column j > 8 is reached only from rows j-4..j+4; columns 0..8 also from the
// wall rows 0..3.
__device__ __forceinline__ double2 ldd(const double2* p) { return *p; }
__device__ __forceinline__ double2 ldd(const float2* p) { return to_d(*p); }  // exact
template <class X2>
__device__ __forceinline__ double2 band_col(const Geo& g, const double* B0, const X2* x, int j, int im, int k) {
    double2 acc = make_double2(0, 0);
    if (j > 8) {
#pragma unroll
        for (int t = -4; t <= 4; ++t) {
            const int c = j + t;
            if (c < g.nr) acc = dfma(__ldg(B0 + (size_t)c * kB + (4 - t)), ldd(x + sidx(g, c, im, k)), acc);
        }
    } else {
#pragma unroll
        for (int t = -8; t <= 4; ++t) {
            const int c = j + t;
            if (c >= 0 && c < g.nr)
                acc = dfma(__ldg(B0 + (size_t)c * kB + (4 - t)), ldd(x + sidx(g, c, im, k)), acc);
        }
    }
    return acc;
}

// vorticity output in FP64, or in FP32 for the mixed-precision transforms,
// which consume it only after rounding to FP32
__device__ __forceinline__ void put_w(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void put_w(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

template <class W2>
__global__ void k_curl(Geo g, const double2* __restrict__ u, W2* __restrict__ w, float2* __restrict__ uf) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    u += d.off;
    w += d.off;
    const double2 *ur = u, *ut = u + d.S, *uz = u + 2 * d.S;
    const double kz = __ldg(g.kzt + d.k), ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    const size_t o = sidx(g, d.j, d.im, d.k);
    const double2 dz = band_row(g, g.D1 + ((size_t)par_idx(d.m) * g.nr + d.j) * kB, uz, d.j, d.im, d.k);
    const double2 dt = band_row(g, g.D1 + ((size_t)par_idx(d.m + 1) * g.nr + d.j) * kB, ut, d.j, d.im, d.k);
    const double2 a = ur[o], b = ut[o], c = uz[o];
    if (uf) {  // u itself rounded to FP32, for the same transforms
        uf += d.off;
        put_w(uf + o, a);
        put_w(uf + o + d.S, b);
        put_w(uf + o + 2 * d.S, c);
    }
    put_w(w + o, make_double2(-mr * c.y + kz * b.y, mr * c.x - kz * b.x));
    put_w(w + o + d.S, make_double2(-kz * a.y - dz.x, kz * a.x - dz.y));
    put_w(w + o + 2 * d.S, make_double2(dt.x + ir * b.x + mr * a.y, dt.y + ir * b.y - mr * a.x));
}

template <class WB2>
__global__ void k_curlT_acc(Geo g, const WB2* __restrict__ wb, double2* __restrict__ ub) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    wb += d.off;
    ub += d.off;
    const WB2 *wr = wb, *wt = wb + d.S, *wz = wb + 2 * d.S;
    const double kz = __ldg(g.kzt + d.k), ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    const size_t o = sidx(g, d.j, d.im, d.k);
    const double2 sT = band_col(g, g.D1 + (size_t)par_idx(d.m + 1) * g.nr * kB, wz, d.j, d.im, d.k);
    const double2 sP = band_col(g, g.D1 + (size_t)par_idx(d.m) * g.nr * kB, wt, d.j, d.im, d.k);
    const double2 a = ldd(wr + o), b = ldd(wt + o), c = ldd(wz + o);
    double2 x = ub[o];
    ub[o] = make_double2(x.x + kz * b.y - mr * c.y, x.y - kz * b.x + mr * c.x);
    x = ub[o + d.S];
    ub[o + d.S] = make_double2(x.x - kz * a.y + sT.x + ir * c.x, x.y + kz * a.x + sT.y + ir * c.y);
    x = ub[o + 2 * d.S];
    ub[o + 2 * d.S] = make_double2(x.x + mr * a.y - sP.x, x.y - mr * a.x - sP.y);
}

__device__ __forceinline__ void base_at(const Geo& g, int slot, int j, double c, double s, double& U, double& dU) {
    const double r = g.r[j];
    const double2 a = g.Uh[(size_t)slot * g.sNr + j], b = g.dUh[(size_t)slot * g.sNr + j];
    U = 1.0 - r * r + (a.x * c - a.y * s);
    dU = -2.0 * r + (b.x * c - b.y * s);
}

// U and dU/dr at the block's radius and batch entry (a spectral block covers
// one j of one entry), at that entry's phase g.cs[b]: one thread evaluates them and
// the block shares the pair, instead of every thread repeating the same FP64
// arithmetic.  Called by all threads of the block before any of them returns.
__device__ __forceinline__ void base_block(const Geo& g, double& U, double& dU) {
    __shared__ double sh[2];
    if (threadIdx.x == 0) {
        const int b = blockIdx.z / g.nr, j = blockIdx.z - b * g.nr;
        const double2 cs = g.cs[b];
        base_at(g, g.slot[b], j, cs.x, cs.y, sh[0], sh[1]);
    }
    __syncthreads();
    U = sh[0];
    dU = sh[1];
}

// N = -U du/dz - u_r dU/dr e_z: the base-flow terms in advective form.  The
// rotational form (U e_z) x w + u x (-dU/dr e_theta) differs from it by
// grad(U u_z), which the discrete pressure projection does not remove exactly;
// the remainder couples u_z back into (u_r, u_theta) and makes k = 0 modes of
// steady pipe flow grow at high Re.
__global__ void k_base(Geo g, const double2* __restrict__ u, double2* __restrict__ N) {
    grid_dep_sync();
    double U, dU;
    base_block(g, U, dU);
    Idx d;
    if (!decode(g, d)) return;
    u += d.off;
    N += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double a = __ldg(g.kzt + d.k) * U;  // -U d/dz = -i a
    const double2 ur = u[o], ut = u[o + S], uz = u[o + 2 * S];
    N[o] = make_double2(a * ur.y, -a * ur.x);
    N[o + S] = make_double2(a * ut.y, -a * ut.x);
    N[o + 2 * S] = make_double2(a * uz.y - dU * ur.x, -a * uz.x - dU * ur.y);
}

// transpose (Euclidean cotangents): ub = conj(-i a) nb = i a nb; ub_r -= dU nb_z
__global__ void k_baseT(Geo g, const double2* __restrict__ nb, double2* __restrict__ ub) {
    grid_dep_sync();
    double U, dU;
    base_block(g, U, dU);
    Idx d;
    if (!decode(g, d)) return;
    nb += d.off;
    ub += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double a = __ldg(g.kzt + d.k) * U;
    const double2 nr_ = nb[o], nt = nb[o + S], nz = nb[o + 2 * S];
    ub[o] = make_double2(-a * nr_.y - dU * nz.x, a * nr_.x - dU * nz.y);
    ub[o + S] = make_double2(-a * nt.y, a * nt.x);
    ub[o + 2 * S] = make_double2(-a * nz.y, a * nz.x);
}

// Velocity-gradient tensor in cylindrical components, G[3 i + j] = (grad u)_ij:
// (d_r u_j), ((im u_r - u_theta)/r, (im u_theta + u_r)/r, im u_z / r), (i k_z u_j).
__global__ void k_grad_u(Geo g, const double2* __restrict__ u, double2* __restrict__ G) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;  // single-request launches only (the launcher checks)
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j), kz = __ldg(g.kzt + d.k);
    const double2 a = u[o], b = u[o + S], c = u[o + 2 * S];
    const double* Bv = g.D1 + ((size_t)par_idx(d.m + 1) * g.nr + d.j) * kB;
    const double* Bz = g.D1 + ((size_t)par_idx(d.m) * g.nr + d.j) * kB;
    G[o] = band_row(g, Bv, u, d.j, d.im, d.k);
    G[o + S] = band_row(g, Bv, u + S, d.j, d.im, d.k);
    G[o + 2 * S] = band_row(g, Bz, u + 2 * S, d.j, d.im, d.k);
    G[o + 3 * S] = make_double2(-mr * a.y - ir * b.x, mr * a.x - ir * b.y);
    G[o + 4 * S] = make_double2(-mr * b.y + ir * a.x, mr * b.x + ir * a.y);
    G[o + 5 * S] = make_double2(-mr * c.y, mr * c.x);
    G[o + 6 * S] = make_double2(-kz * a.y, kz * a.x);
    G[o + 7 * S] = make_double2(-kz * b.y, kz * b.x);
    G[o + 8 * S] = make_double2(-kz * c.y, kz * c.x);
}

// Base-flow part of the continuous-adjoint forcing: N = U dw/dz - w_z dU/dr e_r
__global__ void k_base_adj(Geo g, const double2* __restrict__ w, double2* __restrict__ N) {
    grid_dep_sync();
    double U, dU;
    base_block(g, U, dU);
    Idx d;
    if (!decode(g, d)) return;
    w += d.off;
    N += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double a = __ldg(g.kzt + d.k) * U;  // U d/dz = i a
    const double2 wr = w[o], wt = w[o + S], wz = w[o + 2 * S];
    N[o] = make_double2(-a * wr.y - dU * wz.x, a * wr.x - dU * wz.y);
    N[o + S] = make_double2(-a * wt.y, a * wt.x);
    N[o + 2 * S] = make_double2(-a * wz.y, a * wz.x);
}

// ------------------------------------------------------------------ double-FP32 banded products
// The same products as k_curl, k_curlT_acc, k_stage_div, k_stage_rhs,
// k_stageT_qbar and k_stageT_div, with the band rows and every term carrying
// cancellation accumulated in double-float arithmetic (dev_df.cuh) instead of
// FP64; inputs are split and outputs joined without FP64 instructions but the
// final additions.  Used when the context's precision has the PNOP_DF bit.
struct dacc2 {
    dacc re, im;
};
__device__ __forceinline__ dfl dff(float2 v) {
    dfl r;
    r.h = v.x;
    r.l = v.y;
    return r;
}
__device__ __forceinline__ dacc dacc_neg(dacc a) {
    a.s = -a.s;
    a.c = -a.c;
    return a;
}
__device__ __forceinline__ void df_fma2(dacc2& a, dfl k, const dfc& x) {
    df_fma(a.re, k, x.re);
    df_fma(a.im, k, x.im);
}
// The double-FP32 kernels work on tiles: a block owns kTK consecutive k of
// one m and kTJ consecutive radial rows; it loads the banded input fields on
// rows [j0 - 8, j0 + kTJ + 4) (clipped to the grid; this covers the one-sided
// wall stencils and the transposed columns), splits every value once into
// (hi, lo) pairs in shared memory, and each of its kTG radial groups then
// computes rows j0 + y, j0 + y + kTG, ... from the tile.  A value is split
// about 1.75 times instead of once per band entry that reads it.
constexpr int kTK = 32, kTG = 8, kTJ = 16, kTR = kTJ + 12;
struct TBlk {
    int k, im, m, slot, j0, j1, lo, hi;
    size_t S, off;
    bool on;
};
__device__ __forceinline__ TBlk tdecode(const Geo& g) {
    TBlk t;
    t.S = (size_t)g.nr * g.nm * g.nk;
    t.k = blockIdx.x * kTK + threadIdx.x;
    t.im = blockIdx.y;
    t.m = t.im - g.M;
    const int ntj = (g.nr + kTJ - 1) / kTJ, b = blockIdx.z / ntj, tj = blockIdx.z - b * ntj;
    t.slot = g.slot[b];
    t.off = (size_t)t.slot * g.fs;
    t.j0 = tj * kTJ;
    t.j1 = min(g.nr, t.j0 + kTJ);
    t.lo = max(0, t.j0 - 8);
    t.hi = min(g.nr, t.j0 + kTJ + 4);
    t.on = t.k < g.nk;
    return t;
}
typedef float4 DfTile[kTR][kTK];  // (re.hi, re.lo, im.hi, im.lo) per (row - lo, k)
// a field value as a tile entry: FP64 values are split, an FP32 field is a
// pair with a zero low part
__device__ __forceinline__ float4 tile_entry(double2 v) {
    const dfl re = df_split(v.x), im = df_split(v.y);
    return make_float4(re.h, re.l, im.h, im.l);
}
__device__ __forceinline__ float4 tile_entry(float2 v) { return make_float4(v.x, 0.f, v.y, 0.f); }
template <class F2> __device__ __forceinline__ F2 zero2() {
    F2 z;
    z.x = 0;
    z.y = 0;
    return z;
}
// rows lo + y, lo + y + kTG, ... of one banded field into its tile
template <class F2> __device__ __forceinline__ void tile_load(const Geo& g, const TBlk& t, const F2* f, DfTile& tl) {
    for (int r = t.lo + (int)threadIdx.y; r < t.hi; r += kTG)
        tl[r - t.lo][threadIdx.x] = tile_entry(t.on ? f[sidx(g, r, t.im, t.k)] : zero2<F2>());
}
// The same for two fields, every load of the thread issued before the first
// split: the two-tile kernels (curl and its transpose) measured faster so
// (26.9 against 28.7 ms per gradient), the one-tile kernels did not.
constexpr int kTI = (kTR + kTG - 1) / kTG;  // rows per thread in a tile load
template <class F2>
__device__ __forceinline__ void tile_load2(const Geo& g, const TBlk& t, const F2* f0, DfTile& t0, const F2* f1,
                                           DfTile& t1) {
    F2 raw[2][kTI];
#pragma unroll
    for (int i = 0; i < kTI; ++i) {
        const int r = t.lo + (int)threadIdx.y + i * kTG;
        const bool in = t.on && r < t.hi;
        raw[0][i] = in ? f0[sidx(g, r, t.im, t.k)] : zero2<F2>();
        raw[1][i] = in ? f1[sidx(g, r, t.im, t.k)] : zero2<F2>();
    }
#pragma unroll
    for (int i = 0; i < kTI; ++i) {
        const int r = t.lo + (int)threadIdx.y + i * kTG;
        if (r < t.hi) {
            t0[r - t.lo][threadIdx.x] = tile_entry(raw[0][i]);
            t1[r - t.lo][threadIdx.x] = tile_entry(raw[1][i]);
        }
    }
}
__device__ __forceinline__ dfc df_load(const float2* p) {
    const float2 v = *p;
    dfc r;
    r.re.h = v.x;
    r.re.l = 0.f;
    r.im.h = v.y;
    r.im.l = 0.f;
    return r;
}
__device__ __forceinline__ dfc tile_at(const DfTile& tl, int lo, int r) {
    const float4 v = tl[r - lo][threadIdx.x];
    dfc x;
    x.re.h = v.x;
    x.re.l = v.y;
    x.im.h = v.z;
    x.im.l = v.w;
    return x;
}
// sum_s B[j][s] x[j-4+s] from the tile (rows as in band_row)
__device__ __forceinline__ dacc2 band_row_t(const Geo& g, const float2* B, const DfTile& tl, int lo, int j) {
    dacc2 a{dacc0(), dacc0()};
    if (j >= 4) {
#pragma unroll
        for (int s = 0; s < 9; ++s) {
            const int c = j - 4 + s;
            if (c < g.nr) df_fma2(a, dff(__ldg(B + s)), tile_at(tl, lo, c));
        }
    } else {
#pragma unroll
        for (int s = 0; s < kB; ++s) {
            const int c = j - 4 + s;
            if (c >= 0 && c <= 8) df_fma2(a, dff(__ldg(B + s)), tile_at(tl, lo, c));
        }
    }
    return a;
}
// (B^T x)_j from the tile (columns as in band_col)
__device__ __forceinline__ dacc2 band_col_t(const Geo& g, const float2* B0, const DfTile& tl, int lo, int j) {
    dacc2 a{dacc0(), dacc0()};
    if (j > 8) {
#pragma unroll
        for (int t = -4; t <= 4; ++t) {
            const int c = j + t;
            if (c < g.nr) df_fma2(a, dff(__ldg(B0 + (size_t)c * kB + (4 - t))), tile_at(tl, lo, c));
        }
    } else {
#pragma unroll
        for (int t = -8; t <= 4; ++t) {
            const int c = j + t;
            if (c >= 0 && c < g.nr) df_fma2(a, dff(__ldg(B0 + (size_t)c * kB + (4 - t))), tile_at(tl, lo, c));
        }
    }
    return a;
}
__device__ __forceinline__ double2 df_out(const dacc2& a) { return make_double2(df_result(a.re), df_result(a.im)); }
// the accumulated value rounded once to FP32 (s + c is the rounding of the pair)
__device__ __forceinline__ void df_put(double2* p, const dacc2& a) { *p = df_out(a); }
__device__ __forceinline__ void df_put(float2* p, const dacc2& a) {
    *p = make_float2(a.re.s + a.re.c, a.im.s + a.im.c);
}

// the pair rounded once to FP32
__device__ __forceinline__ float2 df_f32(const dfc& x) { return make_float2(x.re.h + x.re.l, x.im.h + x.im.l); }

template <class W2>
__global__ void __launch_bounds__(kTK* kTG) k_curl_df(Geo g, const double2* __restrict__ u, W2* __restrict__ w,
                                                      float2* __restrict__ uf) {
    grid_dep_sync();
    __shared__ DfTile tz, tt;
    const TBlk t = tdecode(g);
    u += t.off;
    w += t.off;
    const double2 *ur = u, *ut = u + t.S, *uz = u + 2 * t.S;
    tile_load2(g, t, uz, tz, ut, tt);
    __syncthreads();
    if (!t.on) return;
    const dfl kz = dff(__ldg(g.kztf + t.k));
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const dfl ir = dff(__ldg(g.invrf + j)), mr = dff(__ldg(g.mrtf + (size_t)t.im * g.nr + j));
        const size_t o = sidx(g, j, t.im, t.k);
        const dacc2 dz = band_row_t(g, g.D1f + ((size_t)par_idx(t.m) * g.nr + j) * kB, tz, t.lo, j);
        const dacc2 dt = band_row_t(g, g.D1f + ((size_t)par_idx(t.m + 1) * g.nr + j) * kB, tt, t.lo, j);
        const dfc a = df_load(ur + o), b = tile_at(tt, t.lo, j), c = tile_at(tz, t.lo, j);
        dacc2 wr{dacc0(), dacc0()};  // (-mr c.y + kz b.y, mr c.x - kz b.x)
        df_fma(wr.re, df_neg(mr), c.im);
        df_fma(wr.re, kz, b.im);
        df_fma(wr.im, mr, c.re);
        df_fma(wr.im, df_neg(kz), b.re);
        dacc2 wt{dacc_neg(dz.re), dacc_neg(dz.im)};  // (-kz a.y - dz.x, kz a.x - dz.y)
        df_fma(wt.re, df_neg(kz), a.im);
        df_fma(wt.im, kz, a.re);
        dacc2 wz = dt;  // (dt.x + ir b.x + mr a.y, dt.y + ir b.y - mr a.x)
        df_fma(wz.re, ir, b.re);
        df_fma(wz.re, mr, a.im);
        df_fma(wz.im, ir, b.im);
        df_fma(wz.im, df_neg(mr), a.re);
        df_put(w + o, wr);
        df_put(w + o + t.S, wt);
        df_put(w + o + 2 * t.S, wz);
        if (uf) {  // u itself rounded to FP32, for the same transforms
            uf[t.off + o] = df_f32(a);
            uf[t.off + o + t.S] = df_f32(b);
            uf[t.off + o + 2 * t.S] = df_f32(c);
        }
    }
}

template <class WB2>
__global__ void __launch_bounds__(kTK* kTG) k_curlT_acc_df(Geo g, const WB2* __restrict__ wb,
                                                         double2* __restrict__ ub) {
    grid_dep_sync();
    __shared__ DfTile tz, tt;
    const TBlk t = tdecode(g);
    wb += t.off;
    ub += t.off;
    const WB2 *wr = wb, *wt = wb + t.S, *wz = wb + 2 * t.S;
    tile_load2(g, t, wz, tz, wt, tt);
    __syncthreads();
    if (!t.on) return;
    const dfl kz = dff(__ldg(g.kztf + t.k));
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const dfl ir = dff(__ldg(g.invrf + j)), mr = dff(__ldg(g.mrtf + (size_t)t.im * g.nr + j));
        const size_t o = sidx(g, j, t.im, t.k);
        const dacc2 sT = band_col_t(g, g.D1f + (size_t)par_idx(t.m + 1) * g.nr * kB, tz, t.lo, j);
        const dacc2 sP = band_col_t(g, g.D1f + (size_t)par_idx(t.m) * g.nr * kB, tt, t.lo, j);
        const dfc a = df_load(wr + o), b = tile_at(tt, t.lo, j), c = tile_at(tz, t.lo, j);
        dacc2 xr{dacc0(), dacc0()};  // += (kz b.y - mr c.y, -kz b.x + mr c.x)
        df_fma(xr.re, kz, b.im);
        df_fma(xr.re, df_neg(mr), c.im);
        df_fma(xr.im, df_neg(kz), b.re);
        df_fma(xr.im, mr, c.re);
        dacc2 xt = sT;  // += (-kz a.y + sT.x + ir c.x, kz a.x + sT.y + ir c.y)
        df_fma(xt.re, df_neg(kz), a.im);
        df_fma(xt.re, ir, c.re);
        df_fma(xt.im, kz, a.re);
        df_fma(xt.im, ir, c.im);
        dacc2 xz{dacc_neg(sP.re), dacc_neg(sP.im)};  // += (mr a.y - sP.x, -mr a.x - sP.y)
        df_fma(xz.re, mr, a.im);
        df_fma(xz.im, df_neg(mr), a.re);
        double2 x = ub[o], v = df_out(xr);
        ub[o] = make_double2(x.x + v.x, x.y + v.y);
        x = ub[o + t.S];
        v = df_out(xt);
        ub[o + t.S] = make_double2(x.x + v.x, x.y + v.y);
        x = ub[o + 2 * t.S];
        v = df_out(xz);
        ub[o + 2 * t.S] = make_double2(x.x + v.x, x.y + v.y);
    }
}

__global__ void __launch_bounds__(kTK* kTG) k_stage_div_df(Geo g, const double2* __restrict__ F,
                                                         double2* __restrict__ q) {
    grid_dep_sync();
    __shared__ DfTile tr;
    const TBlk t = tdecode(g);
    F += t.off;
    q += t.off;
    tile_load(g, t, F, tr);
    __syncthreads();
    if (!t.on) return;
    const size_t S = t.S;
    const dfl kz = dff(__ldg(g.kztf + t.k));
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const size_t o = sidx(g, j, t.im, t.k);
        if (j == 0 || (t.m == 0 && t.k == 0)) {
            q[o] = make_double2(0, 0);
            continue;
        }
        const dfl ir = dff(__ldg(g.invrf + j)), mr = dff(__ldg(g.mrtf + (size_t)t.im * g.nr + j));
        dacc2 acc = band_row_t(g, g.D1f + ((size_t)par_idx(t.m + 1) * g.nr + j) * kB, tr, t.lo, j);
        const dfc fr = tile_at(tr, t.lo, j), ft = df_load(F + o + S), fz = df_load(F + o + 2 * S);
        df_fma(acc.re, ir, fr.re);  // + ir fr.x - mr ft.y - kz fz.y
        df_fma(acc.re, df_neg(mr), ft.im);
        df_fma(acc.re, df_neg(kz), fz.im);
        df_fma(acc.im, ir, fr.im);  // + ir fr.y + mr ft.x + kz fz.x
        df_fma(acc.im, mr, ft.re);
        df_fma(acc.im, kz, fz.re);
        q[o] = df_out(acc);
    }
}

// k_stage_rhs with every term of R in double-float: R_+ = F_r - F_t i - D1 p
// + (m/r) p ..., written out per real part below
__global__ void __launch_bounds__(kTK* kTG) k_stage_rhs_df(Geo g, const double2* __restrict__ u,
                                                         const double2* __restrict__ F,
                                                         const double2* __restrict__ p, double2* __restrict__ R) {
    grid_dep_sync();
    __shared__ DfTile tp;
    const TBlk t = tdecode(g);
    u = moved(u, t.off);
    F += t.off;
    p += t.off;
    R += t.off;
    tile_load(g, t, p, tp);
    __syncthreads();
    if (!t.on) return;
    const size_t S = t.S;
    const dfl kz = dff(__ldg(g.kztf + t.k));
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const size_t o = sidx(g, j, t.im, t.k);
        if (j == 0) {  // the wall row: T u (no arithmetic worth double-float)
            double2 vp = make_double2(0, 0), vm = vp, vz = vp;
            if (u) {
                const double2 a = u[o], b = u[o + S], c = u[o + 2 * S];
                vp = make_double2(a.x - b.y, a.y + b.x);
                vm = make_double2(a.x + b.y, a.y - b.x);
                vz = c;
            }
            R[o] = vp;
            R[o + S] = vm;
            R[o + 2 * S] = vz;
            continue;
        }
        const dfl mr = dff(__ldg(g.mrtf + (size_t)t.im * g.nr + j));
        const dacc2 dp = band_row_t(g, g.D1f + ((size_t)par_idx(t.m) * g.nr + j) * kB, tp, t.lo, j);
        const dfc pj = tile_at(tp, t.lo, j), fr = df_load(F + o), ft = df_load(F + o + S), fz = df_load(F + o + 2 * S);
        // rp = (Fr.x - Ft.y - dp.x + mr p.x, Fr.y + Ft.x - dp.y + mr p.y)
        // rm = (Fr.x + Ft.y - dp.x - mr p.x, Fr.y - Ft.x - dp.y - mr p.y)
        // rz = (Fz.x + kz p.y, Fz.y - kz p.x)
        dacc2 rp{dacc_neg(dp.re), dacc_neg(dp.im)}, rm = rp, rz{dacc0(), dacc0()};
        df_add(rp.re, fr.re);
        df_add(rp.re, df_neg(ft.im));
        df_fma(rp.re, mr, pj.re);
        df_add(rp.im, fr.im);
        df_add(rp.im, ft.re);
        df_fma(rp.im, mr, pj.im);
        df_add(rm.re, fr.re);
        df_add(rm.re, ft.im);
        df_fma(rm.re, df_neg(mr), pj.re);
        df_add(rm.im, fr.im);
        df_add(rm.im, df_neg(ft.re));
        df_fma(rm.im, df_neg(mr), pj.im);
        df_add(rz.re, fz.re);
        df_fma(rz.re, kz, pj.im);
        df_add(rz.im, fz.im);
        df_fma(rz.im, df_neg(kz), pj.re);
        if (u) {  // + (2/dt) T u: u+ = (a.x - b.y, a.y + b.x), u- = (a.x + b.y, a.y - b.x), u_z
            const dfl f = dff(g.two_dtf[t.slot]);
            const dfc a = df_load(u + o), b = df_load(u + o + S), c = df_load(u + o + 2 * S);
            df_fma(rp.re, f, a.re);
            df_fma(rp.re, df_neg(f), b.im);
            df_fma(rp.im, f, a.im);
            df_fma(rp.im, f, b.re);
            df_fma(rm.re, f, a.re);
            df_fma(rm.re, f, b.im);
            df_fma(rm.im, f, a.im);
            df_fma(rm.im, df_neg(f), b.re);
            df_fma(rz.re, f, c.re);
            df_fma(rz.im, f, c.im);
        }
        R[o] = df_out(rp);
        R[o + S] = df_out(rm);
        R[o + 2 * S] = df_out(rz);
    }
}

__global__ void __launch_bounds__(kTK* kTG) k_stageT_qbar_df(Geo g, const double2* __restrict__ Fb,
                                                           double2* __restrict__ q) {
    grid_dep_sync();
    __shared__ DfTile tr;
    const TBlk t = tdecode(g);
    Fb += t.off;
    q += t.off;
    tile_load(g, t, Fb, tr);
    __syncthreads();
    if (!t.on) return;
    const size_t S = t.S;
    const dfl kz = dff(__ldg(g.kztf + t.k));
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const size_t o = sidx(g, j, t.im, t.k);
        if (t.m == 0 && t.k == 0) {
            q[o] = make_double2(0, 0);
            continue;
        }
        const dfl mr = dff(__ldg(g.mrtf + (size_t)t.im * g.nr + j));
        dacc2 acc = band_col_t(g, g.D1f + (size_t)par_idx(t.m) * g.nr * kB, tr, t.lo, j);
        const dfc ft = df_load(Fb + o + S), fz = df_load(Fb + o + 2 * S);
        df_fma(acc.re, mr, ft.im);  // + mr ft.y + kz fz.y
        df_fma(acc.re, kz, fz.im);
        df_fma(acc.im, df_neg(mr), ft.re);  // - mr ft.x - kz fz.x
        df_fma(acc.im, df_neg(kz), fz.re);
        q[o] = df_out(acc);
    }
}

__global__ void __launch_bounds__(kTK* kTG) k_stageT_div_df(Geo g, const double2* __restrict__ z,
                                                          double2* __restrict__ Fb) {
    grid_dep_sync();
    __shared__ DfTile tz;
    const TBlk t = tdecode(g);
    z += t.off;
    Fb += t.off;
    tile_load(g, t, z, tz);
    __syncthreads();
    if (!t.on || (t.m == 0 && t.k == 0)) return;
    const size_t S = t.S;
    const double kz = __ldg(g.kzt + t.k);
    for (int j = t.j0 + threadIdx.y; j < t.j1; j += kTG) {
        const size_t o = sidx(g, j, t.im, t.k);
        const double mr = __ldg(g.mrt + (size_t)t.im * g.nr + j);
        const dfl ir = dff(__ldg(g.invrf + j));
        dacc2 dz = band_col_t(g, g.D1f + (size_t)par_idx(t.m + 1) * g.nr * kB, tz, t.lo, j);
        const double2 zj = z[o];
        const dfc zd = tile_at(tz, t.lo, j);
        df_fma(dz.re, ir, zd.re);  // D1v^T z + z / r
        df_fma(dz.im, ir, zd.im);
        const double2 v = df_out(dz);
        double2 x = Fb[o];
        Fb[o] = make_double2(x.x - v.x, x.y - v.y);
        x = Fb[o + S];
        Fb[o + S] = make_double2(x.x - mr * zj.y, x.y + mr * zj.x);
        x = Fb[o + 2 * S];
        Fb[o + 2 * S] = make_double2(x.x - kz * zj.y, x.y + kz * zj.x);
    }
}

// ------------------------------------------------------------------ radial stage (forward)
// q = div F (rows j >= 1; q_0 = 0 is the tentative Neumann datum)
__global__ void k_stage_div(Geo g, const double2* __restrict__ F, double2* __restrict__ q) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    F += d.off;
    q += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    if (d.j == 0 || (d.m == 0 && d.k == 0)) {
        q[o] = make_double2(0, 0);
        return;
    }
    const double kz = __ldg(g.kzt + d.k), ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    double2 acc = band_row(g, g.D1 + ((size_t)par_idx(d.m + 1) * g.nr + d.j) * kB, F, d.j, d.im, d.k);
    const double2 fr = F[o], ft = F[o + S], fz = F[o + 2 * S];
    acc.x += ir * fr.x - mr * ft.y - kz * fz.y;
    acc.y += ir * fr.y + mr * ft.x + kz * fz.x;
    q[o] = acc;
}

// ------------------------------------------------------------------ banded solves
// Two-sweep solve of one banded system per (matrix, k) with precomputed
// row-local coefficients "lower | 1/diag | upper" (layout in setup.hpp).  A
// block owns kSK consecutive k of one (component, m) -- one tile of the factor
// table: the right-hand sides of all rows sit in shared memory and the
// coefficient rows stream through a double-buffered cp.async pipeline, kRC
// rows at a time.  In the tiled table the coefficients of kRC consecutive rows
// of one sweep are one contiguous piece, so staging a chunk is a plain linear
// copy.  Each of the 2 kSK threads sweeps the real or the imaginary part of one
// system (the matrices are real).  Terms are accumulated oldest first, so the
// dependence from one row to the next is a single FMA.
constexpr int kRC = 8;        // rows per staged chunk
constexpr int kRegRows = 64;  // grids up to this many radial points keep their columns in registers

__device__ __forceinline__ void cp_async16(void* sm, const void* gm) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(sm);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gm) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// NL lower coefficients (oldest first) for the forward sweep, diagonal in the
// forward sweep when DIAG1 (else in the backward sweep), NU upper coefficients
// (nearest first) for the backward sweep.  X = A^{-1} X [+ add].
// Batch entry blockIdx.y; its factor table sits at fac + slot * fac_stride
// (stride 0: a table shared by all slots).
template <int NL, int NU, bool DIAG1, bool WALL>
__global__ void __launch_bounds__(2 * kSK) k_band_solve(Geo g, const double* __restrict__ fac, size_t fac_stride,
                                                  double2* __restrict__ X, const double2* __restrict__ add, int helm,
                                                  int zero_row0, double* __restrict__ pw,
                                                  const double2* __restrict__ usub) {
    grid_dep_sync();
    constexpr int NC1 = NL + (DIAG1 ? 1 : 0);  // forward sweep: columns [0, NC1)
    constexpr int NC2 = kB - NC1;               // backward sweep: columns [NC1, 13)
    constexpr int NCM = NC1 > NC2 ? NC1 : NC2;
    extern __shared__ __align__(16) unsigned char smem[];
    double2* Yb = reinterpret_cast<double2*>(smem);  // [nr][kSK]
    double* Yd = reinterpret_cast<double*>(smem);
    double* Cb = reinterpret_cast<double*>(Yb + (size_t)g.nr * kSK);  // [2][kRC][NCM][kSK]
    int bi = blockIdx.x;
    const int kb = bi % g.ntile;
    bi /= g.ntile;
    const int im = bi % g.nm, v = bi / g.nm;
    const int m = im - g.M;
    const int mv = helm ? (v == 0 ? m + 1 : (v == 1 ? m - 1 : m)) : m;
    const int k0 = kb * kSK;
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    const int slot = g.slot[blockIdx.y];
    const size_t off = (size_t)slot * g.fs;
    fac += (size_t)slot * fac_stride;
    X += off;
    add = moved(add, off);
    double2* x = X + (size_t)v * S;  // v = 0 for the pressure
    const double* T1 = fac + ((size_t)abs(mv) * g.ntile + kb) * (size_t)g.nr * kB * kSK;  // [nr][NC1][kSK]
    const double* T2 = T1 + (size_t)g.nr * NC1 * kSK;                                    // [nr][NC2][kSK]
    const int tid = threadIdx.x, sy = tid % kSK, comp = tid / kSK;
    const int nch = (g.nr + kRC - 1) / kRC;

    for (int i = tid; i < g.nr * kSK; i += 2 * kSK) {
        const int j = i / kSK, t = i % kSK;
        if (k0 + t < g.nk) cp_async16(&Yb[i], &x[sidx(g, j, im, k0 + t)]);
        else Yb[i] = make_double2(0, 0);
    }
    auto stage = [&](int t) {  // chunk t of the sweep sequence into buffer t & 1
        if (t >= 2 * nch) return;
        const bool fwd = t < nch;
        const int c = fwd ? t : 2 * nch - 1 - t;
        const int rows = min(kRC, g.nr - c * kRC);
        const int nc = fwd ? NC1 : NC2;
        const double* src = (fwd ? T1 : T2) + (size_t)c * kRC * nc * kSK;
        double* dst = Cb + (size_t)(t & 1) * kRC * NCM * kSK;
        const int nseg = rows * nc * (kSK / 2);
        for (int i = tid; i < nseg; i += 2 * kSK) cp_async16(dst + 2 * i, src + 2 * i);
    };
    stage(0);
    cp_async_commit();
    double w1[NL], w2[NU];
#pragma unroll
    for (int e = 0; e < NL; ++e) w1[e] = 0.0;
#pragma unroll
    for (int e = 0; e < NU; ++e) w2[e] = 0.0;
    for (int t = 0; t < 2 * nch; ++t) {
        stage(t + 1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const double* C = Cb + (size_t)(t & 1) * kRC * NCM * kSK + sy;
        if (t < nch) {
#pragma unroll
            for (int r = 0; r < kRC; ++r) {
                const int j = t * kRC + r;
                if (j < g.nr) {
                    double val = Yd[(j * kSK + sy) * 2 + comp];
                    const bool full = !(NL == 8 && j > 8);  // columns of U beyond row 8 hold 4 entries
#pragma unroll
                    for (int e = 0; e < NL; ++e)
                        if (full || e >= NL - 4) val = fma(-C[(r * NC1 + e) * kSK], w1[e], val);
                    if (DIAG1) val *= C[(r * NC1 + NL) * kSK];
#pragma unroll
                    for (int e = 0; e < NL - 1; ++e) w1[e] = w1[e + 1];
                    w1[NL - 1] = val;
                    Yd[(j * kSK + sy) * 2 + comp] = val;
                }
            }
        } else {
            const int c = 2 * nch - 1 - t;
            constexpr int O = DIAG1 ? 0 : 1;  // first upper coefficient of the backward slice
#pragma unroll
            for (int r = kRC - 1; r >= 0; --r) {
                const int j = c * kRC + r;
                if (j < g.nr) {
                    double val = Yd[(j * kSK + sy) * 2 + comp];
                    const bool full = !(NU == 8 && j >= 4);  // rows of U from 4 on hold 4 entries
#pragma unroll
                    for (int e = NU - 1; e >= 0; --e)
                        if (full || e < 4) val = fma(-C[(r * NC2 + O + e) * kSK], w2[e], val);
                    if (!DIAG1) val *= C[(r * NC2) * kSK];
#pragma unroll
                    for (int e = NU - 1; e > 0; --e) w2[e] = w2[e - 1];
                    w2[0] = val;
                    Yd[(j * kSK + sy) * 2 + comp] = val;
                }
            }
        }
        __syncthreads();
    }
    if (WALL && k0 + sy < g.nk) {  // wall partials of the tentative velocity (as in k_band_solve_reg)
        usub = moved(usub, off);
        const double* us = usub ? reinterpret_cast<const double*>(usub) + comp : nullptr;
        double* P = pw + ((((size_t)slot * 3 + v) * g.nm + im) * g.nk + (k0 + sy)) * 2 + comp;
        if (v < 2) {
            const double* d0 = g.D1 + (size_t)par_idx(m + 1) * g.nr * kB + 4;
            double acc = 0.0;
            for (int c = 0; c <= 8 && c < g.nr; ++c) {
                double xv = 0.5 * Yd[(c * kSK + sy) * 2 + comp];
                if (v == 0 && us) xv -= us[2 * sidx(g, c, im, k0 + sy)];
                acc = fma(__ldg(d0 + c), xv, acc);
            }
            *P = acc;
        } else if (m == 0 && k0 + sy == 0) {
            double acc = 0.0;
            for (int j = 0; j < g.nr; ++j) {
                const double xj = Yd[(j * kSK + sy) * 2 + comp];
                acc = fma(g.W[j], us ? xj - us[2 * (2 * S + sidx(g, j, im, 0))] : xj, acc);
            }
            *P = acc;
        }
    }
    for (int i = tid; i < g.nr * kSK; i += 2 * kSK) {
        const int j = i / kSK, t = i % kSK;
        if (k0 + t >= g.nk) continue;
        const size_t o = sidx(g, j, im, k0 + t);
        double2 val = (zero_row0 && j == 0) ? make_double2(0, 0) : Yb[i];
        if (add) {
            const double2 a = add[(size_t)v * S + o];
            val.x += a.x;
            val.y += a.y;
        }
        x[o] = val;
    }
}

// The same two-sweep solve with each thread's column held in registers
// (grids of at most MAXR radial points; the launch bound of six blocks per SM
// keeps the register count at 168, which holds the column without spills).  The column stays in x[0..MAXR): the
// forward sweep reads its lower neighbours and the backward sweep its upper
// neighbours straight from registers (every index is a compile-time constant
// after unrolling), so no shared-memory round trip sits on the dependent
// chain of a row; shared memory holds only the staged coefficient rows.  The
// arithmetic and its order are those of k_band_solve: the results are the
// same to the last bit (up to the sign of zero).
template <int NL, int NU, bool DIAG1, int MAXR, bool WALL>
__global__ void __launch_bounds__(2 * kSK, 6) k_band_solve_reg(Geo g, const double* __restrict__ fac, size_t fac_stride,
                                                      double2* __restrict__ X, const double2* __restrict__ add,
                                                      int helm, int zero_row0, double* __restrict__ pw,
                                                      const double2* __restrict__ usub) {
    grid_dep_sync();
    constexpr int NC1 = NL + (DIAG1 ? 1 : 0);
    constexpr int NC2 = kB - NC1;
    constexpr int NCM = NC1 > NC2 ? NC1 : NC2;
    constexpr int MAXCH = MAXR / kRC;
    static_assert(MAXR % kRC == 0, "whole chunks");
    extern __shared__ __align__(16) unsigned char smem[];
    double* Cb = reinterpret_cast<double*>(smem);  // [2][kRC][NCM][kSK]
    int bi = blockIdx.x;
    const int kb = bi % g.ntile;
    bi /= g.ntile;
    const int im = bi % g.nm, v = bi / g.nm;
    const int m = im - g.M;
    const int mv = helm ? (v == 0 ? m + 1 : (v == 1 ? m - 1 : m)) : m;
    const int k0 = kb * kSK;
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    const int slot = g.slot[blockIdx.y];
    const size_t off = (size_t)slot * g.fs;
    fac += (size_t)slot * fac_stride;
    X += off;
    add = moved(add, off);
    const double* T1 = fac + ((size_t)abs(mv) * g.ntile + kb) * (size_t)g.nr * kB * kSK;
    const double* T2 = T1 + (size_t)g.nr * NC1 * kSK;
    const int tid = threadIdx.x, sy = tid % kSK, comp = tid / kSK;
    const int nr = g.nr, nch = (nr + kRC - 1) / kRC;
    const bool on = k0 + sy < g.nk;
    // this thread's column: the real or imaginary part of system (v, m, k0 + sy)
    const double* xs = reinterpret_cast<const double*>(X + (size_t)v * S) + comp;
    double x[MAXR];
#pragma unroll
    for (int j = 0; j < MAXR; ++j) x[j] = (on && j < nr) ? xs[2 * sidx(g, j, im, k0 + sy)] : 0.0;
    // wall partials of the tentative velocity T^-1 x - usub (forward Helmholtz
    // solves): the usub part now, the solution's part after the sweeps.
    // v = 0, 1: d0 . (x/2) over rows 0..8 (d0 the wall row of D1 for u_r), minus
    // d0 . usub_r on v = 0; the mean mode's u_z block: sum_j W_j (x - usub_z).
    const bool mean_z = v == 2 && m == 0 && k0 + sy == 0;
    double wall_u = 0.0;
    if (WALL && on && usub) {
        const double* us = reinterpret_cast<const double*>(usub + off) + comp;
        if (v == 0) {
            const double* d0 = g.D1 + (size_t)par_idx(m + 1) * nr * kB + 4;
#pragma unroll 1
            for (int c = 0; c <= 8 && c < nr; ++c) wall_u = fma(__ldg(d0 + c), us[2 * sidx(g, c, im, k0 + sy)], wall_u);
        } else if (mean_z) {
#pragma unroll 1
            for (int j = 0; j < nr; ++j) wall_u = fma(g.W[j], us[2 * (2 * S + sidx(g, j, im, 0))], wall_u);
        }
    }
    auto stage = [&](int t) {  // chunk t of the sweep sequence into buffer t & 1
        if (t >= 2 * nch) return;
        const bool fwd = t < nch;
        const int c = fwd ? t : 2 * nch - 1 - t;
        const int rows = min(kRC, nr - c * kRC);
        const int nc = fwd ? NC1 : NC2;
        const double* src = (fwd ? T1 : T2) + (size_t)c * kRC * nc * kSK;
        double* dst = Cb + (size_t)(t & 1) * kRC * NCM * kSK;
        const int nseg = rows * nc * (kSK / 2);
        for (int i = tid; i < nseg; i += 2 * kSK) cp_async16(dst + 2 * i, src + 2 * i);
    };
    stage(0);
    cp_async_commit();
#pragma unroll
    for (int t = 0; t < MAXCH; ++t) {
        if (t < nch) {
            stage(t + 1);
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            const double* C = Cb + (size_t)(t & 1) * kRC * NCM * kSK + sy;
#pragma unroll
            for (int r = 0; r < kRC; ++r) {
                const int j = t * kRC + r;
                if (j < nr) {
                    double val = x[j];
                    const bool full = !(NL == 8 && j > 8);
#pragma unroll
                    for (int e = 0; e < NL; ++e) {
                        const int jj = j - NL + e;  // w1[e] of k_band_solve: oldest first
                        if (jj >= 0 && (full || e >= NL - 4)) val = fma(-C[(r * NC1 + e) * kSK], x[jj >= 0 ? jj : 0], val);
                    }
                    if (DIAG1) val *= C[(r * NC1 + NL) * kSK];
                    x[j] = val;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int c = MAXCH - 1; c >= 0; --c) {
        if (c < nch) {
            const int t = 2 * nch - 1 - c;
            stage(t + 1);
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            const double* C = Cb + (size_t)(t & 1) * kRC * NCM * kSK + sy;
            constexpr int O = DIAG1 ? 0 : 1;
#pragma unroll
            for (int r = kRC - 1; r >= 0; --r) {
                const int j = c * kRC + r;
                if (j < nr) {
                    double val = x[j];
                    const bool full = !(NU == 8 && j >= 4);
#pragma unroll
                    for (int e = NU - 1; e >= 0; --e) {
                        const int jj = j + 1 + e;  // w2[e] of k_band_solve: nearest first (0 beyond nr)
                        if (jj < MAXR && (full || e < 4)) val = fma(-C[(r * NC2 + O + e) * kSK], x[jj < MAXR ? jj : 0], val);
                    }
                    if (!DIAG1) val *= C[(r * NC2) * kSK];
                    x[j] = val;
                }
            }
            __syncthreads();
        }
    }
    if (!on) return;
    if (WALL) {
        double* P = pw + ((((size_t)slot * 3 + v) * g.nm + im) * g.nk + (k0 + sy)) * 2 + comp;
        if (v < 2) {
            const double* d0 = g.D1 + (size_t)par_idx(m + 1) * nr * kB + 4;
            double acc = 0.0;
#pragma unroll
            for (int c = 0; c <= 8; ++c)
                if (c < nr) acc = fma(__ldg(d0 + c), 0.5 * x[c], acc);
            *P = acc - wall_u;
        } else if (mean_z) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < MAXR; ++j)
                if (j < nr) acc = fma(g.W[j], x[j], acc);
            *P = acc - wall_u;
        }
    }
    double* xo = reinterpret_cast<double*>(X + (size_t)v * S) + comp;
    const double* ad = add ? reinterpret_cast<const double*>(add + (size_t)v * S) + comp : nullptr;
#pragma unroll
    for (int j = 0; j < MAXR; ++j) {
        if (j < nr) {
            const size_t o = 2 * sidx(g, j, im, k0 + sy);
            double val = (zero_row0 && j == 0) ? 0.0 : x[j];
            if (ad) val += ad[o];
            xo[o] = val;
        }
    }
}

// R_v = F'_v [+ (2/dt) (T u)_v] for v = +, -, z (rows j >= 1), F' = F - grad p;
// wall row R_v = (T u)_v (0 without u).  T u: u+ = u_r + i u_theta,
// u- = u_r - i u_theta, u_z.  With A_v + B_v = 2 I / dt this right-hand side
// gives A_v^{-1} E (B_v T u + F') + T u.
__global__ void k_stage_rhs(Geo g, const double2* __restrict__ u, const double2* __restrict__ F,
                            const double2* __restrict__ p, double2* __restrict__ R) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    u = moved(u, d.off);
    F += d.off;
    p += d.off;
    R += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    double2 tp = make_double2(0, 0), tm = tp, tz = tp;
    if (u) {
        const double2 a = u[o], b = u[o + S], c = u[o + 2 * S];
        tp = make_double2(a.x - b.y, a.y + b.x);
        tm = make_double2(a.x + b.y, a.y - b.x);
        tz = c;
    }
    if (d.j == 0) {
        R[o] = tp;
        R[o + S] = tm;
        R[o + 2 * S] = tz;
        return;
    }
    const double kz = __ldg(g.kzt + d.k), mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    const double2 dp = band_row(g, g.D1 + ((size_t)par_idx(d.m) * g.nr + d.j) * kB, p, d.j, d.im, d.k);
    const double2 pj = p[o], fr0 = F[o], ft0 = F[o + S], fz0 = F[o + 2 * S];
    const double2 fr = make_double2(fr0.x - dp.x, fr0.y - dp.y);
    const double2 ft = make_double2(ft0.x + mr * pj.y, ft0.y - mr * pj.x);
    const double2 fz = make_double2(fz0.x + kz * pj.y, fz0.y - kz * pj.x);
    double2 rp = make_double2(fr.x - ft.y, fr.y + ft.x), rm = make_double2(fr.x + ft.y, fr.y - ft.x), rz = fz;
    if (u) {
        const double f = g.two_dt[d.slot];
        rp = dfma(f, tp, rp);
        rm = dfma(f, tm, rm);
        rz = dfma(f, tz, rz);
    }
    R[o] = rp;
    R[o + S] = rm;
    R[o + 2 * S] = rz;
}

// Per-mode kernels of the wall conditions run on blocks of kFK consecutive k
// (x) times kFJ radial groups (y) of one m: a per-mode scalar is reduced over
// j into shared memory in a fixed order (deterministic), then every thread
// applies it to its rows j = y, y + kFJ, ...  Fields and the influence table
// are k-fastest, so a warp reads 32 consecutive k of one row.
constexpr int kFK = 32, kFJ = 8;
// influence response component c (0: u_r, 1: u_theta / i, 2: u_z / i) at row j of mode (im, k)
__device__ __forceinline__ double infl_at(const double* h, const Geo& g, int im, int c, int j, int k) {
    return __ldg(h + (((size_t)im * 3 + c) * g.nr + j) * g.nk + k);
}

// out = [addto +] back to (r, theta, z) [- usub] with the influence
// correction (div u = 0 at the wall) or, for mode (0,0), flux correction and
// u_r = 0, one value per thread.  The mode's coefficient comes from the wall
// partials the Helmholtz solve left in pw ([slot][3][m][k]): a0 = pw[0] +
// pw[1] = d/dr u_r at the wall of the tentative velocity
// u_r = (x+ + x-)/2 [- usub_r], or for mode (0,0) pw[2] = sum_j W_j
// (x_z [- usub_z]).
__global__ void k_stage_finish(Geo g, const double2* __restrict__ R, const double2* __restrict__ addto,
                               const double2* __restrict__ usub, const double2* __restrict__ pw,
                               double2* __restrict__ out) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    R += d.off;
    addto = moved(addto, d.off);
    usub = moved(usub, d.off);
    out += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S, nmk = (size_t)g.nm * g.nk;
    const bool mean = d.m == 0 && d.k == 0;
    const double2* P = pw + (size_t)d.slot * 3 * nmk + (size_t)d.im * g.nk + d.k;
    double2 a0;
    if (mean) {
        a0 = P[2 * nmk];
    } else {
        const double2 p0 = P[0], p1 = P[nmk];
        a0 = make_double2(p0.x + p1.x, p0.y + p1.y);
    }
    const double2 xp = R[o], xm = R[o + S];
    double2 ur = make_double2(0.5 * (xp.x + xm.x), 0.5 * (xp.y + xm.y));
    double2 ut = make_double2(0.5 * (xp.y - xm.y), -0.5 * (xp.x - xm.x));
    double2 uz = R[o + 2 * S];
    if (usub) {
        const double2 a = usub[o], b = usub[o + S], c = usub[o + 2 * S];
        ur.x -= a.x; ur.y -= a.y;
        ut.x -= b.x; ut.y -= b.y;
        uz.x -= c.x; uz.y -= c.y;
    }
    if (mean) {
        uz = dfma(slot_fluxg(g, d.slot)[d.j] * (-g.flux_inv[d.slot]), a0, uz);
        ur = make_double2(0, 0);
    } else {
        const double* h = slot_infl(g, d.slot);
        const double h0 = infl_at(h, g, d.im, 0, d.j, d.k), h1 = infl_at(h, g, d.im, 1, d.j, d.k),
                     h2 = infl_at(h, g, d.im, 2, d.j, d.k);
        ur = dfma(h0, a0, ur);
        ut = make_double2(ut.x - h1 * a0.y, ut.y + h1 * a0.x);
        uz = make_double2(uz.x - h2 * a0.y, uz.y + h2 * a0.x);
    }
    if (addto) {
        const double2 a = addto[o], b = addto[o + S], c = addto[o + 2 * S];
        ur.x += a.x; ur.y += a.y;
        ut.x += b.x; ut.y += b.y;
        uz.x += c.x; uz.y += c.y;
    }
    out[o] = ur;
    out[o + S] = ut;
    out[o + 2 * S] = uz;
}

// k_stage_finish in double-float arithmetic (PNOP_DF): the same combination
// with one FP64 addition per output part
__global__ void k_stage_finish_df(Geo g, const double2* __restrict__ R, const double2* __restrict__ addto,
                                  const double2* __restrict__ usub, const double2* __restrict__ pw,
                                  double2* __restrict__ out) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    R += d.off;
    addto = moved(addto, d.off);
    usub = moved(usub, d.off);
    out += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S, nmk = (size_t)g.nm * g.nk;
    const bool mean = d.m == 0 && d.k == 0;
    const double2* P = pw + (size_t)d.slot * 3 * nmk + (size_t)d.im * g.nk + d.k;
    dfc a0;
    if (mean) {
        a0 = df_load(P + 2 * nmk);
    } else {
        const dfc p0 = df_load(P), p1 = df_load(P + nmk);
        dacc s0 = dacc0(), s1 = dacc0();
        df_add(s0, p0.re);
        df_add(s0, p1.re);
        df_add(s1, p0.im);
        df_add(s1, p1.im);
        a0.re = df_val(s0);
        a0.im = df_val(s1);
    }
    const dfc xp = df_load(R + o), xm = df_load(R + o + S), xz = df_load(R + o + 2 * S);
    dfl half;
    half.h = 0.5f;
    half.l = 0.f;
    // u_r = (x+ + x-)/2, u_theta = (x+ - x-)/(2i), u_z
    dacc2 ur{dacc0(), dacc0()}, ut{dacc0(), dacc0()}, uz{dacc0(), dacc0()};
    df_fma(ur.re, half, xp.re);
    df_fma(ur.re, half, xm.re);
    df_fma(ur.im, half, xp.im);
    df_fma(ur.im, half, xm.im);
    df_fma(ut.re, half, xp.im);
    df_fma(ut.re, df_neg(half), xm.im);
    df_fma(ut.im, df_neg(half), xp.re);
    df_fma(ut.im, half, xm.re);
    df_add(uz.re, xz.re);
    df_add(uz.im, xz.im);
    if (usub) {
        const dfc a = df_load(usub + o), b = df_load(usub + o + S), c = df_load(usub + o + 2 * S);
        df_add(ur.re, df_neg(a.re));
        df_add(ur.im, df_neg(a.im));
        df_add(ut.re, df_neg(b.re));
        df_add(ut.im, df_neg(b.im));
        df_add(uz.re, df_neg(c.re));
        df_add(uz.im, df_neg(c.im));
    }
    if (mean) {
        const dfl f = df_split(slot_fluxg(g, d.slot)[d.j] * (-g.flux_inv[d.slot]));
        df_fma(uz.re, f, a0.re);
        df_fma(uz.im, f, a0.im);
        ur = dacc2{dacc0(), dacc0()};
    } else {
        const double* h = slot_infl(g, d.slot);
        const dfl h0 = df_split(infl_at(h, g, d.im, 0, d.j, d.k)), h1 = df_split(infl_at(h, g, d.im, 1, d.j, d.k)),
                  h2 = df_split(infl_at(h, g, d.im, 2, d.j, d.k));
        df_fma(ur.re, h0, a0.re);
        df_fma(ur.im, h0, a0.im);
        df_fma(ut.re, df_neg(h1), a0.im);  // ut += i h1 a0
        df_fma(ut.im, h1, a0.re);
        df_fma(uz.re, df_neg(h2), a0.im);
        df_fma(uz.im, h2, a0.re);
    }
    if (addto) {
        const dfc a = df_load(addto + o), b = df_load(addto + o + S), c = df_load(addto + o + 2 * S);
        df_add(ur.re, a.re);
        df_add(ur.im, a.im);
        df_add(ut.re, b.re);
        df_add(ut.im, b.im);
        df_add(uz.re, c.re);
        df_add(uz.im, c.im);
    }
    out[o] = df_out(ur);
    out[o + S] = df_out(ut);
    out[o + 2 * S] = df_out(uz);
}

// ------------------------------------------------------------------ radial stage (transpose)
// Per mode: ybar = Fin^H ubar_new (a reduction over j), then xbar = Ti^H ybar.
// The mode's coefficient acc of Fin^H goes to ac (added to it when ac_add), so
// that Fin^H can be applied again later without the reduction.
__global__ void __launch_bounds__(kFK* kFJ) k_stageT_finish(Geo g, const double2* __restrict__ un,
                                                           double2* __restrict__ R, double2* __restrict__ ac,
                                                           int ac_add) {
    grid_dep_sync();
    __shared__ double2 red[kFJ][kFK];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int k = blockIdx.x * kFK + tx, im = blockIdx.y, m = im - g.M;
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    const int slot = g.slot[blockIdx.z];  // batch entry blockIdx.z
    const size_t off = (size_t)slot * g.fs;
    un += off;
    R += off;
    const bool on = k < g.nk, mean = (m == 0 && k == 0);
    const double* h = slot_infl(g, slot);
    const double* fg = slot_fluxg(g, slot);
    double2 part = make_double2(0, 0);
    if (on) {
        for (int j = ty; j < g.nr; j += kFJ) {
            const size_t o = sidx(g, j, im, k);
            if (mean) {
                part = dfma(fg[j], un[o + 2 * S], part);
            } else {
                const double2 a = un[o], b = un[o + S], c = un[o + 2 * S];
                const double h0 = infl_at(h, g, im, 0, j, k), h1 = infl_at(h, g, im, 1, j, k),
                             h2 = infl_at(h, g, im, 2, j, k);
                // infl0 a - i infl1 b - i infl2 c
                part.x += h0 * a.x + h1 * b.y + h2 * c.y;
                part.y += h0 * a.y - h1 * b.x - h2 * c.x;
            }
        }
    }
    red[ty][tx] = part;
    __syncthreads();
    if (!on) return;
    double2 acc = red[0][tx];
#pragma unroll
    for (int i = 1; i < kFJ; ++i) acc = make_double2(acc.x + red[i][tx].x, acc.y + red[i][tx].y);
    if (ty == 0) {
        double2* a = ac + ((size_t)slot * g.nm + im) * g.nk + k;
        if (ac_add) {
            const double2 prev = *a;
            *a = make_double2(prev.x + acc.x, prev.y + acc.y);
        } else {
            *a = acc;
        }
    }
    const double* d0 = g.D1 + (size_t)par_idx(m + 1) * g.nr * kB;
    for (int j = ty; j < g.nr; j += kFJ) {
        const size_t o = sidx(g, j, im, k);
        double2 yr = un[o], yt = un[o + S], yz = un[o + 2 * S];
        if (mean) {
            yr = make_double2(0, 0);
            yz = dfma(-g.flux_inv[slot] * g.W[j], acc, yz);
        } else if (j <= 8) {
            yr = dfma(__ldg(d0 + 4 + j), acc, yr);
        }
        R[o] = make_double2(0.5 * (yr.x - yt.y), 0.5 * (yr.y + yt.x));
        R[o + S] = make_double2(0.5 * (yr.x + yt.y), 0.5 * (yr.y - yt.x));
        R[o + 2 * S] = yz;
    }
}

// With X = Z = A^{-T} T^-H Fin^H v (wall row kept) and E the projection on
// rows j >= 1:
//   ub (=, or += when acc) T^H ((2/dt) E Z + e0 Z_0) - Fin^H v  when ub is given,
//     v = V1 [+ V2], Fin^H v from the stored per-mode coefficients ac
//     (u_r rows 0..8 gain d0_j ac; mode (0,0): u_r = 0, u_z gains
//     -flux_inv W_j ac): the transpose of the velocity part of the stage;
//   Fb = T^H E (cf1 X + cf2 Y)  when Fb is given (Y is read only when TWO).
template <bool TWO>
__global__ void k_stageT_rhs(Geo g, const double2* __restrict__ X, const double2* __restrict__ Y, double cf1,
                             double cf2, double2* __restrict__ ub, int acc, double2* __restrict__ Fb,
                             const double2* __restrict__ V1, const double2* __restrict__ V2,
                             const double2* __restrict__ ac) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    X += d.off;
    Y = moved(Y, d.off);
    ub = moved(ub, d.off);
    Fb = moved(Fb, d.off);
    V1 = moved(V1, d.off);
    V2 = moved(V2, d.off);
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double2 rp = X[o], rm = X[o + S], rz = X[o + 2 * S];
    if (ub) {
        const double f = d.j == 0 ? 1.0 : g.two_dt[d.slot];
        const double2 bp = dscale(rp, f), bm = dscale(rm, f), bz = dscale(rz, f);
        double2 vr = make_double2(bp.x + bm.x, bp.y + bm.y);
        double2 vt = make_double2(bp.y - bm.y, -bp.x + bm.x);
        double2 vz = bz;
        double2 mr = V1[o], mt = V1[o + S], mz = V1[o + 2 * S];
        if (V2) {
            const double2 a = V2[o], b = V2[o + S], c = V2[o + 2 * S];
            mr.x += a.x; mr.y += a.y;
            mt.x += b.x; mt.y += b.y;
            mz.x += c.x; mz.y += c.y;
        }
        const double2 cm = ac[((size_t)d.slot * g.nm + d.im) * g.nk + d.k];
        if (d.m == 0 && d.k == 0) {
            mr = make_double2(0, 0);
            mz = dfma(-g.flux_inv[d.slot] * g.W[d.j], cm, mz);
        } else if (d.j <= 8) {
            mr = dfma(__ldg(g.D1 + (size_t)par_idx(d.m + 1) * g.nr * kB + 4 + d.j), cm, mr);
        }
        vr.x -= mr.x; vr.y -= mr.y;
        vt.x -= mt.x; vt.y -= mt.y;
        vz.x -= mz.x; vz.y -= mz.y;
        if (acc) {
            const double2 a = ub[o], b = ub[o + S], c = ub[o + 2 * S];
            vr.x += a.x; vr.y += a.y;
            vt.x += b.x; vt.y += b.y;
            vz.x += c.x; vz.y += c.y;
        }
        ub[o] = vr;
        ub[o + S] = vt;
        ub[o + 2 * S] = vz;
    }
    if (Fb) {
        if (d.j == 0) {
            Fb[o] = Fb[o + S] = Fb[o + 2 * S] = make_double2(0, 0);
            return;
        }
        double2 p = make_double2(cf1 * rp.x, cf1 * rp.y), q = make_double2(cf1 * rm.x, cf1 * rm.y),
                z = make_double2(cf1 * rz.x, cf1 * rz.y);
        if (TWO) {
            const double2 a = Y[o], b = Y[o + S], c = Y[o + 2 * S];
            p = make_double2(fma(cf2, a.x, p.x), fma(cf2, a.y, p.y));
            q = make_double2(fma(cf2, b.x, q.x), fma(cf2, b.y, q.y));
            z = make_double2(fma(cf2, c.x, z.x), fma(cf2, c.y, z.y));
        }
        Fb[o] = make_double2(p.x + q.x, p.y + q.y);
        Fb[o + S] = make_double2(p.y - q.y, -p.x + q.x);
        Fb[o + 2 * S] = z;
    }
}

// k_stageT_rhs in double-float arithmetic (PNOP_DF): the same outputs with
// every sum and scaling in double-FP32 and one FP64 addition per output part
template <bool TWO>
__global__ void k_stageT_rhs_df(Geo g, const double2* __restrict__ X, const double2* __restrict__ Y, double cf1,
                                double cf2, double2* __restrict__ ub, int acc, double2* __restrict__ Fb,
                                const double2* __restrict__ V1, const double2* __restrict__ V2,
                                const double2* __restrict__ ac) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    X += d.off;
    Y = moved(Y, d.off);
    ub = moved(ub, d.off);
    Fb = moved(Fb, d.off);
    V1 = moved(V1, d.off);
    V2 = moved(V2, d.off);
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const dfc rp = df_load(X + o), rm = df_load(X + o + S), rz = df_load(X + o + 2 * S);
    if (ub) {
        dfl f;
        f.h = 1.f;
        f.l = 0.f;
        if (d.j != 0) f = dff(g.two_dtf[d.slot]);
        // T^H (f rp, f rm, f rz) - Fin^H (V1 + V2): r = f (rp + rm), theta = f (i... ) as in k_stageT_rhs
        dacc2 vr{dacc0(), dacc0()}, vt{dacc0(), dacc0()}, vz{dacc0(), dacc0()};
        df_fma(vr.re, f, rp.re);
        df_fma(vr.re, f, rm.re);
        df_fma(vr.im, f, rp.im);
        df_fma(vr.im, f, rm.im);
        df_fma(vt.re, f, rp.im);
        df_fma(vt.re, df_neg(f), rm.im);
        df_fma(vt.im, df_neg(f), rp.re);
        df_fma(vt.im, f, rm.re);
        df_fma(vz.re, f, rz.re);
        df_fma(vz.im, f, rz.im);
        const dfc a = df_load(V1 + o), b = df_load(V1 + o + S), c = df_load(V1 + o + 2 * S);
        const bool mean = d.m == 0 && d.k == 0;
        if (!mean) {
            df_add(vr.re, df_neg(a.re));
            df_add(vr.im, df_neg(a.im));
        }
        df_add(vt.re, df_neg(b.re));
        df_add(vt.im, df_neg(b.im));
        df_add(vz.re, df_neg(c.re));
        df_add(vz.im, df_neg(c.im));
        if (V2) {
            const dfc a2 = df_load(V2 + o), b2 = df_load(V2 + o + S), c2 = df_load(V2 + o + 2 * S);
            if (!mean) {
                df_add(vr.re, df_neg(a2.re));
                df_add(vr.im, df_neg(a2.im));
            }
            df_add(vt.re, df_neg(b2.re));
            df_add(vt.im, df_neg(b2.im));
            df_add(vz.re, df_neg(c2.re));
            df_add(vz.im, df_neg(c2.im));
        }
        const double2 cm = ac[((size_t)d.slot * g.nm + d.im) * g.nk + d.k];
        if (mean) {  // Fin^H: u_r = 0, u_z gains -flux_inv W_j cm
            const dfl kf = df_split(g.flux_inv[d.slot] * g.W[d.j]);
            df_fma(vz.re, kf, df_split(cm.x));
            df_fma(vz.im, kf, df_split(cm.y));
        } else if (d.j <= 8) {  // Fin^H: u_r rows 0..8 gain d0_j cm
            const dfl kd = df_split(__ldg(g.D1 + (size_t)par_idx(d.m + 1) * g.nr * kB + 4 + d.j));
            df_fma(vr.re, df_neg(kd), df_split(cm.x));
            df_fma(vr.im, df_neg(kd), df_split(cm.y));
        }
        double2 outr = df_out(vr), outt = df_out(vt), outz = df_out(vz);
        if (acc) {
            const double2 pa = ub[o], pb = ub[o + S], pc = ub[o + 2 * S];
            outr = make_double2(outr.x + pa.x, outr.y + pa.y);
            outt = make_double2(outt.x + pb.x, outt.y + pb.y);
            outz = make_double2(outz.x + pc.x, outz.y + pc.y);
        }
        ub[o] = outr;
        ub[o + S] = outt;
        ub[o + 2 * S] = outz;
    }
    if (Fb) {
        if (d.j == 0) {
            Fb[o] = Fb[o + S] = Fb[o + 2 * S] = make_double2(0, 0);
            return;
        }
        const dfl k1 = df_split(cf1);
        dacc2 p{dacc0(), dacc0()}, q{dacc0(), dacc0()}, z{dacc0(), dacc0()};
        df_fma(p.re, k1, rp.re);
        df_fma(p.im, k1, rp.im);
        df_fma(q.re, k1, rm.re);
        df_fma(q.im, k1, rm.im);
        df_fma(z.re, k1, rz.re);
        df_fma(z.im, k1, rz.im);
        if (TWO) {
            const dfl k2 = df_split(cf2);
            const dfc ya = df_load(Y + o), yb = df_load(Y + o + S), yc = df_load(Y + o + 2 * S);
            df_fma(p.re, k2, ya.re);
            df_fma(p.im, k2, ya.im);
            df_fma(q.re, k2, yb.re);
            df_fma(q.im, k2, yb.im);
            df_fma(z.re, k2, yc.re);
            df_fma(z.im, k2, yc.im);
        }
        // (p + q, (p.y - q.y, -p.x + q.x), z)
        const dfl pr = df_val(p.re), pi = df_val(p.im), qr = df_val(q.re), qi = df_val(q.im);
        dacc2 fr{dacc0(), dacc0()}, ft{dacc0(), dacc0()};
        df_add(fr.re, pr);
        df_add(fr.re, qr);
        df_add(fr.im, pi);
        df_add(fr.im, qi);
        df_add(ft.re, pi);
        df_add(ft.re, df_neg(qi));
        df_add(ft.im, df_neg(pr));
        df_add(ft.im, qr);
        Fb[o] = df_out(fr);
        Fb[o + S] = df_out(ft);
        Fb[o + 2 * S] = df_out(z);
    }
}

// qbar = G^H Fb' = D1p^T Fb'_r - i (m/r) Fb'_t - i kz Fb'_z
__global__ void k_stageT_qbar(Geo g, const double2* __restrict__ Fb, double2* __restrict__ q) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    Fb += d.off;
    q += d.off;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    if (d.m == 0 && d.k == 0) {
        q[o] = make_double2(0, 0);
        return;
    }
    const double kz = __ldg(g.kzt + d.k), mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    double2 acc = band_col(g, g.D1 + (size_t)par_idx(d.m) * g.nr * kB, Fb, d.j, d.im, d.k);
    const double2 ft = Fb[o + S], fz = Fb[o + 2 * S];
    acc.x += mr * ft.y + kz * fz.y;
    acc.y += -mr * ft.x - kz * fz.x;
    q[o] = acc;
}

// Fb = Fb' - Dv^H z: Fb_r -= D1v^T z + z/r ; Fb_t += i (m/r) z ; Fb_z += i kz z
__global__ void k_stageT_div(Geo g, const double2* __restrict__ z, double2* __restrict__ Fb) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    z += d.off;
    Fb += d.off;
    if (d.m == 0 && d.k == 0) return;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    const double kz = __ldg(g.kzt + d.k), ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j);
    const double2 dz = band_col(g, g.D1 + (size_t)par_idx(d.m + 1) * g.nr * kB, z, d.j, d.im, d.k);
    const double2 zj = z[o];
    double2 x = Fb[o];
    Fb[o] = make_double2(x.x - dz.x - ir * zj.x, x.y - dz.y - ir * zj.y);
    x = Fb[o + S];
    Fb[o + S] = make_double2(x.x - mr * zj.y, x.y + mr * zj.x);
    x = Fb[o + 2 * S];
    Fb[o + 2 * S] = make_double2(x.x - kz * zj.y, x.y + kz * zj.x);
}

// ------------------------------------------------------------------ admissible projection
// Orthogonal projection onto admissible fields in the energy inner product:
// Hermitian k = 0 plane, no slip, discrete divergence zero at every r_j, and
// for the mean mode u_r = 0 with zero flux.  Per mode (m, k) != (0, 0):
// y = C x (wall values removed), solve S z = y (S = C W^-1 C^H, real SPD,
// banded Cholesky factors), x -= W^-1 C^H z.

// u(m, 0) and u(-m, 0) <- their Hermitian average; one thread per (c, j, m >= 0)
__global__ void k_proj_herm(Geo g, double2* __restrict__ u) {
    grid_dep_sync();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * g.nr * (g.M + 1)) return;
    const int m = t % (g.M + 1), cj = t / (g.M + 1);
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    const int c = cj / g.nr, j = cj % g.nr;
    double2* a = u + c * S + sidx(g, j, g.M + m, 0);
    double2* b = u + c * S + sidx(g, j, g.M - m, 0);
    const double2 p = *a, q = *b;
    const double2 h = make_double2(0.5 * (p.x + q.x), 0.5 * (p.y - q.y));
    *a = h;
    *b = make_double2(h.x, -h.y);
}

// y_j = sum_{c >= 1} D1[j][c] u_r[c] + u_r[j] / r_j + (i m / r_j) u_theta[j] + i k_z u_z[j]  (wall values excluded)
__global__ void k_proj_div(Geo g, const double2* __restrict__ u, double2* __restrict__ y) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    if (d.m == 0 && d.k == 0) {
        y[o] = make_double2(0, 0);
        return;
    }
    const double* B = g.D1 + ((size_t)par_idx(d.m + 1) * g.nr + d.j) * kB;
    double2 acc = make_double2(0, 0);
    for (int s = 0; s < kB; ++s) {
        const int c = d.j - 4 + s;
        if (c >= 1 && c < g.nr) acc = dfma(__ldg(B + s), u[sidx(g, c, d.im, d.k)], acc);
    }
    if (d.j >= 1) {
        const double ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j), kz = __ldg(g.kzt + d.k);
        const double2 a = u[o], b = u[o + S], c = u[o + 2 * S];
        acc.x += ir * a.x - mr * b.y - kz * c.y;
        acc.y += ir * a.y + mr * b.x + kz * c.x;
    }
    y[o] = acc;
}

// S z = y in place per mode (one thread per mode and real/imaginary part); the
// mean-mode threads store the W-weighted mean of u_z over j >= 1 in y(0, mean).
__global__ void k_proj_solve(Geo g, const double* __restrict__ L, const double2* __restrict__ u,
                             double2* __restrict__ y) {
    grid_dep_sync();
    constexpr int B = 12, W1 = B + 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * g.nm * g.nk) return;
    const int part = t / (g.nm * g.nk), mode = t % (g.nm * g.nk);
    const int im = mode / g.nk, k = mode % g.nk, m = im - g.M;
    double* Y = reinterpret_cast<double*>(y) + part;
    auto at = [&](int j) -> double& { return Y[2 * sidx(g, j, im, k)]; };
    if (m == 0 && k == 0) {
        const double* uz = reinterpret_cast<const double*>(u + 2 * (size_t)g.nr * g.nm * g.nk) + part;
        double num = 0, den = 0;
        for (int j = 1; j < g.nr; ++j) {
            num += g.W[j] * uz[2 * sidx(g, j, im, k)];
            den += g.W[j];
        }
        at(0) = num / den;
        return;
    }
    const double* F = L + (((size_t)abs(m) * g.nk + k) * g.nr) * W1;
    for (int j = 0; j < g.nr; ++j) {  // L w = y
        double v = at(j);
        for (int i = max(0, j - B); i < j; ++i) v -= F[j * W1 + (i - j + B)] * at(i);
        at(j) = v * F[j * W1 + B];
    }
    for (int j = g.nr - 1; j >= 0; --j) {  // L^T z = w
        double v = at(j);
        for (int i = j + 1; i <= min(g.nr - 1, j + B); ++i) v -= F[i * W1 + (j - i + B)] * at(i);
        at(j) = v * F[j * W1 + B];
    }
}

// u -= W^-1 C^H z; wall values zero; mean mode: u_r = 0, u_z -= its weighted mean
__global__ void k_proj_update(Geo g, double2* __restrict__ u, const double2* __restrict__ z) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    const size_t o = sidx(g, d.j, d.im, d.k), S = d.S;
    if (d.j == 0) {
        u[o] = u[o + S] = u[o + 2 * S] = make_double2(0, 0);
        return;
    }
    if (d.m == 0 && d.k == 0) {
        const double2 mu = z[sidx(g, 0, d.im, d.k)];
        u[o] = make_double2(0, 0);
        const double2 c = u[o + 2 * S];
        u[o + 2 * S] = make_double2(c.x - mu.x, c.y - mu.y);
        return;
    }
    const double ir = g.invr[d.j], mr = __ldg(g.mrt + (size_t)d.im * g.nr + d.j), kz = __ldg(g.kzt + d.k), wi = 1.0 / g.W[d.j];
    const double2 zj = z[o];
    double2 dr = band_col(g, g.D1 + (size_t)par_idx(d.m + 1) * g.nr * kB, z, d.j, d.im, d.k);
    dr.x += ir * zj.x;
    dr.y += ir * zj.y;
    const double2 a = u[o], b = u[o + S], c = u[o + 2 * S];
    u[o] = make_double2(a.x - wi * dr.x, a.y - wi * dr.y);
    u[o + S] = make_double2(b.x - wi * mr * zj.y, b.y + wi * mr * zj.x);
    u[o + 2 * S] = make_double2(c.x - wi * kz * zj.y, c.y + wi * kz * zj.x);
}

// ------------------------------------------------------------------ diagnostics
// Energy of every Fourier mode, split into the cross-section (u_r, u_theta)
// and axial (u_z) parts: E[0][im][k], E[1][im][k] with the weights of the
// energy inner product (2 pi Lz W_j c_k / 2).  One thread per mode, fixed
// summation order.
__global__ void k_mode_energy(Geo g, const double2* __restrict__ u, double* __restrict__ E) {
    grid_dep_sync();
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= g.nm * g.nk) return;
    const int im = mode / g.nk, k = mode % g.nk;
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    double a = 0, b = 0;
    for (int j = 0; j < g.nr; ++j) {
        const size_t o = sidx(g, j, im, k);
        const double2 p = u[o], q = u[o + S], c = u[o + 2 * S];
        a += g.W[j] * (p.x * p.x + p.y * p.y + q.x * q.x + q.y * q.y);
        b += g.W[j] * (c.x * c.x + c.y * c.y);
    }
    const double w = 0.5 * g.ewt * (k == 0 ? 1.0 : 2.0);
    E[mode] = w * a;
    E[g.nm * g.nk + mode] = w * b;
}

// Resolution measures of Section 2.4 in one block, fixed summation order:
// out[0] = energy of the azimuthal mode m = M over the full spectrum
// k = -K..K, out[1] = energy of the axial mode k = K over m = -M..M.  A
// stored mode (m, k > 0) holds e(m, k) + e(-m, -k), so the full-spectrum
// energy of (M, k) is half of stored (M, k) and that of (M, -k) half of
// stored (-M, k); (M, 0) counts once.  For K = 0 the axial mode is k = 0 and
// every stored (m, 0) counts once.
__global__ void __launch_bounds__(1024) k_resolution(Geo g, const double2* __restrict__ u, double* __restrict__ out) {
    grid_dep_sync();
    __shared__ double red[2][1024];
    const size_t S = (size_t)g.nr * g.nm * g.nk;
    const double w0 = 0.5 * g.ewt;
    double aM = 0, aK = 0;
    const int nM = 2 * 3 * g.nr * g.nk;  // (side, c, j, k) with side 0: m = M, side 1: m = -M
    for (int i = threadIdx.x; i < nM; i += blockDim.x) {
        const int k = i % g.nk, rest = i / g.nk, j = rest % g.nr, c = (rest / g.nr) % 3, side = rest / (3 * g.nr);
        // full-spectrum weight: w0 W_j for (M, k >= 0) from side 0 and for
        // (M, -k), k > 0, from side 1 (half the stored weight 2 w0 W_j of a
        // k > 0 mode); stored (-M, 0) is (M, 0)'s conjugate, already counted
        if (side && k == 0) continue;
        const int im = side ? 0 : 2 * g.M;
        const double2 v = u[c * S + sidx(g, j, im, k)];
        aM += w0 * g.W[j] * (v.x * v.x + v.y * v.y);
    }
    const int nK = 3 * g.nr * g.nm;  // (c, j, m) at k = K: full-spectrum weight w0 W_j, K = 0 or not
    for (int i = threadIdx.x; i < nK; i += blockDim.x) {
        const int im = i % g.nm, rest = i / g.nm, j = rest % g.nr, c = rest / g.nr;
        const double2 v = u[c * S + sidx(g, j, im, g.K)];
        aK += w0 * g.W[j] * (v.x * v.x + v.y * v.y);
    }
    red[0][threadIdx.x] = aM;
    red[1][threadIdx.x] = aK;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
    }
}

// ------------------------------------------------------------------ elementwise / reductions
// n values of batch entry blockIdx.y
__global__ void k_axpby(Geo g, size_t n, double a, const double2* __restrict__ x, double b,
                        const double2* __restrict__ y, double2* __restrict__ out) {
    grid_dep_sync();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t off = (size_t)g.slot[blockIdx.y] * g.fs;
    x += off;
    y = moved(y, off);
    out += off;
    const double2 p = x[i];
    double2 r = make_double2(a * p.x, a * p.y);
    if (y) {
        const double2 q = y[i];
        r.x += b * q.x;
        r.y += b * q.y;
    }
    out[i] = r;
}

__global__ void k_weight(Geo g, const double2* __restrict__ x, double2* __restrict__ out, int divide) {
    grid_dep_sync();
    Idx d;
    if (!decode(g, d)) return;
    x += d.off;
    out += d.off;
    const double w = g.ewt * g.W[d.j] * (d.k == 0 ? 1.0 : 2.0);
    const double f = divide ? 1.0 / w : w;
    for (int c = 0; c < 3; ++c) {
        const size_t i = c * d.S + sidx(g, d.j, d.im, d.k);
        out[i] = make_double2(x[i].x * f, x[i].y * f);
    }
}

// One partial per block of the 3-D spectral grid (fixed order: deterministic).
__global__ void k_inner_partial(Geo g, const double2* __restrict__ a, const double2* __restrict__ b,
                                double* __restrict__ partial) {
    grid_dep_sync();
    __shared__ double red[128];
    Idx d;
    double acc = 0;
    if (decode(g, d)) {
        a += d.off;
        b += d.off;
        const double w = g.W[d.j] * (d.k == 0 ? 1.0 : 2.0);
        for (int c = 0; c < 3; ++c) {
            const size_t i = c * d.S + sidx(g, d.j, d.im, d.k);
            const double2 p = a[i], q = b[i];
            acc += w * (p.x * q.x + p.y * q.y);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

// Block b sums the np partials of batch entry b into out[slot[b]].
__global__ void k_inner_final(Geo g, const double* __restrict__ partial, int np, double scale,
                              double* __restrict__ out) {
    grid_dep_sync();
    __shared__ double red[1024];
    double acc = 0;
    partial += (size_t)blockIdx.x * np;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[g.slot[blockIdx.x]] = red[0] * scale;
}

// x *= sqrt(E0 / (scale e2[slot])) over the 3 S values of batch entry blockIdx.y
__global__ void k_scale_energy(Geo g, size_t n, double2* __restrict__ x, double E0, double scale,
                               const double* __restrict__ e2) {
    grid_dep_sync();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = g.slot[blockIdx.y];
    const double f = sqrt(E0 / (scale * e2[slot]));
    x += (size_t)slot * g.fs;
    x[i] = make_double2(f * x[i].x, f * x[i].y);
}

// ------------------------------------------------------------------ launchers
// grid and block of the tiled double-FP32 kernels (x: k tiles, y: m, z: row tiles x batch entries)
static inline dim3 tile_grid(const Geo& g) {
    return dim3((g.nk + kTK - 1) / kTK, g.nm, ((g.nr + kTJ - 1) / kTJ) * g.nb);
}
static inline dim3 tile_block() { return dim3(kTK, kTG); }
// block and grid of the 3-D spectral launches (x: k, y: m, z: r)
static inline unsigned spec_bx(const Geo& g) { return g.nk <= 32 ? 32u : (g.nk <= 64 ? 64u : 128u); }
static inline dim3 spec_grid(const Geo& g) {
    return dim3((g.nk + spec_bx(g) - 1) / spec_bx(g), g.nm, g.nr * g.nb);
}
// Operators that only single-request contexts use (continuous adjoint,
// projection, diagnostics) index no slot: refuse a batched geometry.
static void single_only(const Geo& g, const char* what) {
    if (g.nb != 1 || g.slot[0] != 0)
        throw std::runtime_error(std::string(what) + ": not available on batched launches");
}

template <class W2> static void curl_any(const Geo& g, const double2* u, W2* w, float2* uf, cudaStream_t s) {
    if (g.df) launch_pdl(k_curl_df<W2>, tile_grid(g), tile_block(), 0, s, g, u, w, uf);
    else launch_pdl(k_curl<W2>, spec_grid(g), spec_bx(g), 0, s, g, u, w, uf);
    check_launch("curl");
}
void launch_curl(const Geo& g, const double2* u, double2* w, cudaStream_t s) { curl_any(g, u, w, nullptr, s); }
void launch_curl_f32(const Geo& g, const double2* u, float2* w, float2* uf, cudaStream_t s) {
    curl_any(g, u, w, uf, s);
}
template <class WB2> static void curlT_any(const Geo& g, const WB2* wb, double2* ub, cudaStream_t s) {
    if (g.df) launch_pdl(k_curlT_acc_df<WB2>, tile_grid(g), tile_block(), 0, s, g, wb, ub);
    else launch_pdl(k_curlT_acc<WB2>, spec_grid(g), spec_bx(g), 0, s, g, wb, ub);
    check_launch("curlT");
}
void launch_curlT_acc(const Geo& g, const double2* wb, double2* ub, cudaStream_t s) { curlT_any(g, wb, ub, s); }
void launch_curlT_acc_f32(const Geo& g, const float2* wb, double2* ub, cudaStream_t s) { curlT_any(g, wb, ub, s); }
void launch_grad_u(const Geo& g, const double2* u, double2* G, cudaStream_t s) {
    single_only(g, "grad_u");
    launch_pdl(k_grad_u, spec_grid(g), spec_bx(g), 0, s, g, u, G);
    check_launch("grad_u");
}
void launch_base_adj(const Geo& g, const double2* w, double2* N, cudaStream_t s) {
    launch_pdl(k_base_adj, spec_grid(g), spec_bx(g), 0, s, g, w, N);
    check_launch("base_adj");
}
void launch_base(const Geo& g, const double2* u, double2* N, cudaStream_t s) {
    launch_pdl(k_base, spec_grid(g), spec_bx(g), 0, s, g, u, N);
    check_launch("base");
}
void launch_baseT(const Geo& g, const double2* nb, double2* ub, cudaStream_t s) {
    launch_pdl(k_baseT, spec_grid(g), spec_bx(g), 0, s, g, nb, ub);
    check_launch("baseT");
}

// trans selects the transposed coefficient layout; zero_row0 writes 0 to the
// wall row of the solution; pw (forward Helmholtz solves only) receives the
// wall partials of the tentative velocity, with usub subtracted
static void launch_band_solve(const Geo& g, const double* fac, size_t fac_stride, double2* X, const double2* add,
                              int helm, int trans, int zero_row0, cudaStream_t s, double* pw = nullptr,
                              const double2* usub = nullptr) {
    const dim3 nblocks((unsigned)((helm ? 3 : 1) * g.nm * g.ntile), (unsigned)g.nb);
    // columns in registers for the Helmholtz solves (three systems per mode:
    // several warps per scheduler hide the dependent chain); the pressure
    // solve, one system per mode and about one warp per scheduler, keeps the
    // shared-memory form, which measured faster there.  Only the forward
    // Helmholtz instance carries the wall-partial epilogue (pw).
    if (helm && g.nr <= kRegRows) {
        const size_t sm = 2 * (size_t)kRC * 9 * kSK * sizeof(double);
        auto go = [&](auto kernel, double* wall_pw, const double2* wall_u) {
            smem_limit((const void*)kernel);
            launch_serial(kernel, nblocks, 2 * kSK, sm, s, g, fac, fac_stride, X, add, helm, zero_row0, wall_pw,
                          wall_u);
        };
        if (!trans && pw) go(k_band_solve_reg<4, 8, false, kRegRows, true>, pw, usub);
        else if (!trans) go(k_band_solve_reg<4, 8, false, kRegRows, false>, nullptr, nullptr);
        else go(k_band_solve_reg<8, 4, true, kRegRows, false>, nullptr, nullptr);
        return;
    }
    const size_t sm = (size_t)g.nr * kSK * sizeof(double2) + 2 * (size_t)kRC * 9 * kSK * sizeof(double);
    auto go = [&](auto kernel, double* wall_pw, const double2* wall_u) {
        smem_limit((const void*)kernel);
        launch_serial(kernel, nblocks, 2 * kSK, sm, s, g, fac, fac_stride, X, add, helm, zero_row0, wall_pw, wall_u);
    };
    if (!trans && pw) go(k_band_solve<4, 8, false, true>, pw, usub);
    else if (!trans) go(k_band_solve<4, 8, false, false>, nullptr, nullptr);
    else go(k_band_solve<8, 4, true, false>, nullptr, nullptr);
}

void launch_stage_div(const Geo& g, const double2* F, double2* q, cudaStream_t s) {
    if (g.df) launch_pdl(k_stage_div_df, tile_grid(g), tile_block(), 0, s, g, F, q);
    else launch_pdl(k_stage_div, spec_grid(g), spec_bx(g), 0, s, g, F, q);
    check_launch("stage_div");
}
void launch_stage_psolve(const Geo& g, double2* q, cudaStream_t s) {
    launch_band_solve(g, g.facP, 0, q, nullptr, 0, 0, 0, s);
    check_launch("stage_psolve");
}
void launch_stage_rhs(const Geo& g, const double2* u, const double2* F, const double2* p, double2* R, cudaStream_t s) {
    if (g.df) launch_pdl(k_stage_rhs_df, tile_grid(g), tile_block(), 0, s, g, u, F, p, R);
    else launch_pdl(k_stage_rhs, spec_grid(g), spec_bx(g), 0, s, g, u, F, p, R);
    check_launch("stage_rhs");
}
void launch_stage_hsolve(const Geo& g, double2* R, const double2* usub, double* pw, cudaStream_t s) {
    launch_band_solve(g, g.facH, g.sFacH, R, nullptr, 1, 0, 0, s, pw, usub);
    check_launch("stage_hsolve");
}
static inline dim3 mode_grid(const Geo& g) { return dim3((g.nk + kFK - 1) / kFK, g.nm, g.nb); }
void launch_stage_finish(const Geo& g, const double2* R, const double2* addto, const double2* usub, const double* pw,
                         double2* out, cudaStream_t s) {
    const double2* p2 = reinterpret_cast<const double2*>(pw);
    if (g.df) launch_pdl(k_stage_finish_df, spec_grid(g), spec_bx(g), 0, s, g, R, addto, usub, p2, out);
    else launch_pdl(k_stage_finish, spec_grid(g), spec_bx(g), 0, s, g, R, addto, usub, p2, out);
    check_launch("stage_finish");
}
void launch_stageT_finish(const Geo& g, const double2* ubn, double2* R, double2* ac, int ac_add, cudaStream_t s) {
    launch_serial(k_stageT_finish, mode_grid(g), dim3(kFK, kFJ), 0, s, g, ubn, R, ac, ac_add);
    check_launch("stageT_finish");
}
void launch_stageT_hsolve(const Geo& g, double2* R, const double2* add, cudaStream_t s) {
    launch_band_solve(g, g.facHT, g.sFacH, R, add, 1, 1, 0, s);
    check_launch("stageT_hsolve");
}
void launch_stageT_rhs(const Geo& g, const double2* X, const double2* Y, double cf1, double cf2, double2* ub, int acc,
                       double2* Fb, const double2* V1, const double2* V2, const double2* ac, cudaStream_t s) {
    if (ub && (!V1 || !ac)) throw std::runtime_error("stageT_rhs: the velocity part needs its input and coefficients");
    if (g.df) {
        if (Y)
            launch_pdl(k_stageT_rhs_df<true>, spec_grid(g), spec_bx(g), 0, s, g, X, Y, cf1, cf2, ub, acc, Fb, V1, V2,
                       ac);
        else
            launch_pdl(k_stageT_rhs_df<false>, spec_grid(g), spec_bx(g), 0, s, g, X, Y, cf1, cf2, ub, acc, Fb, V1, V2,
                       ac);
    } else if (Y) {
        launch_pdl(k_stageT_rhs<true>, spec_grid(g), spec_bx(g), 0, s, g, X, Y, cf1, cf2, ub, acc, Fb, V1, V2, ac);
    } else {
        launch_pdl(k_stageT_rhs<false>, spec_grid(g), spec_bx(g), 0, s, g, X, Y, cf1, cf2, ub, acc, Fb, V1, V2, ac);
    }
    check_launch("stageT_rhs");
}
void launch_stageT_qbar(const Geo& g, const double2* Fb, double2* q, cudaStream_t s) {
    if (g.df) launch_pdl(k_stageT_qbar_df, tile_grid(g), tile_block(), 0, s, g, Fb, q);
    else launch_pdl(k_stageT_qbar, spec_grid(g), spec_bx(g), 0, s, g, Fb, q);
    check_launch("stageT_qbar");
}
void launch_stageT_psolve(const Geo& g, double2* q, cudaStream_t s) {
    launch_band_solve(g, g.facPT, 0, q, nullptr, 0, 1, 1, s);
    check_launch("stageT_psolve");
}
void launch_stageT_div(const Geo& g, const double2* z, double2* Fb, cudaStream_t s) {
    if (g.df) launch_pdl(k_stageT_div_df, tile_grid(g), tile_block(), 0, s, g, z, Fb);
    else launch_pdl(k_stageT_div, spec_grid(g), spec_bx(g), 0, s, g, z, Fb);
    check_launch("stageT_div");
}

void launch_mode_energy(const Geo& g, const double2* u, double* E, cudaStream_t s) {
    single_only(g, "mode_energy");
    launch_pdl(k_mode_energy, nblk((size_t)g.nm * g.nk, 128), 128, 0, s, g, u, E);
    check_launch("mode_energy");
}

void launch_resolution(const Geo& g, const double2* u, double* out, cudaStream_t s) {
    single_only(g, "resolution");
    launch_pdl(k_resolution, 1, 1024, 0, s, g, u, out);
    check_launch("resolution");
}

void launch_project(const Geo& g, double2* u, double2* y, const double* L, cudaStream_t s) {
    single_only(g, "project");
    launch_pdl(k_proj_herm, nblk((size_t)3 * g.nr * (g.M + 1), 128), 128, 0, s, g, u);
    launch_pdl(k_proj_div, spec_grid(g), spec_bx(g), 0, s, g, u, y);
    launch_pdl(k_proj_solve, nblk((size_t)2 * g.nm * g.nk, 64), 64, 0, s, g, L, u, y);
    launch_pdl(k_proj_update, spec_grid(g), spec_bx(g), 0, s, g, u, y);
    check_launch("project");
}

void launch_axpby(const Geo& g, size_t n, double a, const double2* x, double b, const double2* y, double2* out,
                  cudaStream_t s) {
    launch_pdl(k_axpby, dim3(nblk(n, 256), g.nb), 256, 0, s, g, n, a, x, b, y, out);
    check_launch("axpby");
}
void launch_weight(const Geo& g, const double2* x, double2* out, int divide, cudaStream_t s) {
    launch_pdl(k_weight, spec_grid(g), spec_bx(g), 0, s, g, x, out, divide);
    check_launch("weight");
}
size_t inner_partials(const Geo& g) {
    const dim3 grid = spec_grid(g);
    return (size_t)grid.x * grid.y * grid.z;
}
void launch_inner(const Geo& g, const double2* a, const double2* b, double* partial, double* dev_out, cudaStream_t s) {
    const dim3 grid = spec_grid(g);
    launch_pdl(k_inner_partial, grid, spec_bx(g), 0, s, g, a, b, partial);
    launch_pdl(k_inner_final, g.nb, 1024, 0, s, g, partial, (int)(grid.x * grid.y * (grid.z / g.nb)), g.ewt, dev_out);
    check_launch("inner");
}
void launch_scale_energy(const Geo& g, double2* x, double E0, double scale, const double* e2, cudaStream_t s) {
    const size_t n = 3 * (size_t)g.nr * g.nm * g.nk;
    launch_pdl(k_scale_energy, dim3(nblk(n, 256), g.nb), 256, 0, s, g, n, x, E0, scale, e2);
    check_launch("scale_energy");
}

}  // namespace pnop
