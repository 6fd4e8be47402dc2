// Device kernels of the forward/adjoint pipe-flow step and their launchers.
#pragma once

#include <cuda_runtime.h>

namespace pnop {

// Systems per banded-solver block: consecutive k of one (component, m).  The
// factor tables are tiled in k by the same count.
constexpr int kSK = 32;

// Most requests one batched launch covers (one storage slot each).
constexpr int kMaxBatch = 16;

// Read-only geometry and operators, passed to kernels by value.
struct Geo {
    int nr, M, K, nm, nk, nt, nzp;
    double kz0;      // 2 pi / Lz
    const double* r;
    const double* invr;
    const double* W;
    const double* D1;    // [2][nr][13]
    const double* Lb;    // [M+2][nr][13]  L_m / (2 Re), no k_z^2 (that sits in dgt)
    int ntile;           // k tiles of kSK values in the factor tables
    const double* facH;  // M+2 Helmholtz matrices, A x = b rows, tiled (4 forward | 9 backward columns)
    const double* facP;  // M+1 pressure matrices, same layout
    const double* facHT; // transposed-solve rows, tiled (9 forward | 4 backward columns)
    const double* facPT;
    const double* infl;  // [nm][3][nr][nk] (k fastest)
    const double* fluxg; // [nr]
    const double2* Uh;   // [nr]
    const double2* dUh;  // [nr]
    double ewt;          // 2 pi Lz (energy weight prefactor)
    // per-mode constants as tables, so that spectral kernels spend no FP64
    // instruction on integer conversions: k_z = k kz0 [nk], m / r_j [nm][nr],
    // 1/dt - k_z^2 / (2 Re) (the explicit Crank-Nicolson diagonal) [nk]
    const double* kzt;
    const double* mrt;
    const double* dgt;
    // Batched launches.  A launch covers nb requests; entry b works on storage
    // slot slot[b].  Every spectral buffer holds one field per slot, slot s at
    // element s * fs; every physical scratch buffer one set of planes per slot
    // at s * ps.  The tables that depend on the request's Re, dt, Wo and A
    // (Lb, facH, facHT, infl, fluxg, Uh, dUh, dgt) hold one copy per slot at
    // the strides below; r, W, D1, facP, facPT, kzt, mrt and the twiddles
    // depend on the grid only and are shared.  A single-request context has
    // nb = 1 and slot[0] = 0, so no pointer moves.
    int nb;
    int slot[kMaxBatch];
    size_t fs, ps;
    size_t sLb, sFacH, sInfl, sNr, sNk;
    double two_dt[kMaxBatch];    // 2 / dt per slot (A + B = 2 I / dt of the Crank-Nicolson pair)
    double flux_inv[kMaxBatch];  // flux normalisation per slot
    double2 cs[kMaxBatch];       // (cos, sin) of the pulsation phase of entry b at the launch's time
    // double-FP32 arithmetic for the explicit banded products (df != 0): the
    // tables as (hi, lo) float pairs, D1 [2][nr][13], 1/r [nr], k_z [nk],
    // m/r [nm][nr], and 2/dt per slot
    int df;
    const float2* D1f;
    const float2* invrf;
    const float2* kztf;
    const float2* mrtf;
    float2 two_dtf[kMaxBatch];
};

// Up to 18 input / 6 output spectral component planes for the transforms; the
// analysis adds add[i] (when not null) to output i.
constexpr int kMaxIn = 18;
struct FieldPtrs {
    const double2* in[kMaxIn];
    const float2* inf[kMaxIn];  // non-null: input field stored in FP32 (in[] unused)
    double2* out[6];
    float2* outf[6];  // non-null: output written in FP32 (out[] unused, add[] must be null)
    const double2* add[6];
};

// Per-field multipliers applied when forming the Hermitian z spectrum:
// H_0 = h0 * Re(Y_0), H_k = hk * Y_k (k >= 1); per-output k-scales o0, ok.
struct ZScales {
    double h0[kMaxIn], hk[kMaxIn];
    double o0[6], ok[6];
    float fh0[kMaxIn], fhk[kMaxIn], fo0[6], fok[6];  // FP32 copies, filled by launch_zpass
};

// Twiddle tables e^{-2 pi i n / N} for N = nt and N = nzp, FP64 and FP32.
struct Twiddles {
    const double2* th_d;
    const double2* z_d;
    const float2* th_f;
    const float2* z_f;
};

// ZFWD: u, w -> u x w (6 -> 3 fields); ZADJ: u, w, g -> w x g, g x u (9 -> 6),
// the transpose; ZCADJ: u, curl w, w, grad u -> -u x curl w - 2 (grad u) . w
// (18 -> 3), the perturbation forcing of the continuous adjoint.
enum ZMode { ZFWD = 0, ZADJ = 1, ZCADJ = 2 };

// ---- spectral FP64 kernels ----
void launch_curl(const Geo& g, const double2* u, double2* w, cudaStream_t s);
// the same vorticity rounded to FP32 (input of the mixed-precision
// transforms), and u itself rounded to FP32 into uf when uf is not null
void launch_curl_f32(const Geo& g, const double2* u, float2* w, float2* uf, cudaStream_t s);
void launch_curlT_acc(const Geo& g, const double2* wb, double2* ub, cudaStream_t s);
// the same with wb stored in FP32
void launch_curlT_acc_f32(const Geo& g, const float2* wb, double2* ub, cudaStream_t s);
// continuous adjoint: G[3 i + j] = (grad u)_ij (9 component planes, i the
// derivative direction), and the base-flow part of its forcing
// Nb = U dw/dz - w_z dU/dr e_r (written)
void launch_grad_u(const Geo& g, const double2* u, double2* G, cudaStream_t s);
void launch_base_adj(const Geo& g, const double2* w, double2* N, cudaStream_t s);
// base-flow terms in advective form: N = -U du/dz - u_r dU/dr e_z, and their
// transpose ub = (dN/du)^T nb (both written, not accumulated), at the phase
// g.cs[b] of each batch entry
void launch_base(const Geo& g, const double2* u, double2* N, cudaStream_t s);
void launch_baseT(const Geo& g, const double2* nb, double2* ub, cudaStream_t s);

// ---- transforms (T = double for FP64, float for mixed) ----
template <class T2>
void launch_synth_theta(const Geo& g, const FieldPtrs& f, int nfield, T2* Y, const Twiddles& tw, cudaStream_t s);
template <class T2>
void launch_zpass(const Geo& g, int mode, const T2* Y, T2* Z, const ZScales& sc, const Twiddles& tw, cudaStream_t s);
template <class T2>
void launch_anal_theta(const Geo& g, const FieldPtrs& f, int nfield, const T2* Z, const Twiddles& tw, cudaStream_t s);

// ---- radial stage (forward): out = S(u, F) ----
// q = div F; p = A_p^{-1} q; R = (F - grad p)_pm [+ (2/dt) T u, wall row T u];
// R = A_v^{-1} R; out = back to (r, theta, z) [- u] + influence / flux
// corrections (Section 2.4).  The explicit Crank-Nicolson half enters through
// A + B = 2 I / dt: A^{-1} E (B u + F) = A^{-1} (2 E u / dt + e0 u_0 + E F) - u,
// so no banded product with the old velocity is formed.
void launch_stage_div(const Geo& g, const double2* F, double2* q, cudaStream_t s);
void launch_stage_psolve(const Geo& g, double2* q, cudaStream_t s);
// R = (F - grad p) in the +/- basis, plus (2/dt) T u (rows j >= 1) and T u
// (wall row) when u is given (u null: forcing-only stage S(0, F))
void launch_stage_rhs(const Geo& g, const double2* u, const double2* F, const double2* p, double2* R, cudaStream_t s);
// R = A_v^{-1} R; its epilogue writes the wall partials of the tentative
// velocity (R back to (r, theta, z), usub subtracted when given) to pw
// ([slot][3][nm][nk] complex): pw[0] + pw[1] = d/dr u_r at the wall,
// pw[2](m = 0, k = 0) = the flux sum_j W_j u_z
void launch_stage_hsolve(const Geo& g, double2* R, const double2* usub, double* pw, cudaStream_t s);
// out = [addto +] finished stage (addto may be null), with the old velocity
// usub subtracted from the tentative velocity when given, and the influence
// (or, for mode (0,0), flux) correction driven by the wall partials pw
void launch_stage_finish(const Geo& g, const double2* R, const double2* addto, const double2* usub, const double* pw,
                         double2* out, cudaStream_t s);
// ---- radial stage (transpose): ub (=, or += when acc) S_u^H ubn, Fb = S_F^H ubn ----
// R = T^-H Fin^H ubn; the per-mode coefficient of Fin^H to ac[slot][m][k]
// (added to what ac holds when ac_add)
void launch_stageT_finish(const Geo& g, const double2* ubn, double2* R, double2* ac, int ac_add, cudaStream_t s);
// R = A^{-T} R [+ add] (add may be null); the wall row is kept
void launch_stageT_hsolve(const Geo& g, double2* R, const double2* add, cudaStream_t s);
// with Z = A^{-T} T^-H Fin^H v (X, the transposed solve's output, E: rows j >= 1):
// ub (=, or += when acc) T^H ((2/dt) E Z + e0 Z_0) - Fin^H v if ub, v = V1 [+ V2]
// (Fin^H from the coefficients ac);  Fb = T^H E (cf1 X + cf2 Y) if Fb (Y may be null)
void launch_stageT_rhs(const Geo& g, const double2* X, const double2* Y, double cf1, double cf2, double2* ub, int acc,
                       double2* Fb, const double2* V1, const double2* V2, const double2* ac, cudaStream_t s);
void launch_stageT_qbar(const Geo& g, const double2* Fb, double2* q, cudaStream_t s);
void launch_stageT_psolve(const Geo& g, double2* q, cudaStream_t s);
void launch_stageT_div(const Geo& g, const double2* z, double2* Fb, cudaStream_t s);

// ---- diagnostics: per-mode energy, E[0] cross-section and E[1] axial parts, [2][nm][nk] ----
void launch_mode_energy(const Geo& g, const double2* u, double* E, cudaStream_t s);
// ---- resolution measures: out[0] energy of m = M (all k), out[1] energy of k = K (all m), full spectrum ----
void launch_resolution(const Geo& g, const double2* u, double* out, cudaStream_t s);

// ---- admissible projection (energy-orthogonal, Section 2.2 constraints) ----
// u <- P u in place; y: one-component scratch field; L: factors of build_projection
void launch_project(const Geo& g, double2* u, double2* y, const double* L, cudaStream_t s);

// ---- elementwise / reductions ----
// out = a x + b y over n values per batch entry (y may be null)
void launch_axpby(const Geo& g, size_t n, double a, const double2* x, double b, const double2* y, double2* out,
                  cudaStream_t s);
void launch_weight(const Geo& g, const double2* x, double2* out, int divide, cudaStream_t s);
// Deterministic weighted inner product sum W_hat Re(conj(a) b); the result of
// batch entry b to dev_out[slot[b]].  partial must hold inner_partials(g)
// doubles (one per block, fixed order).
void launch_inner(const Geo& g, const double2* a, const double2* b, double* partial, double* dev_out, cudaStream_t s);
size_t inner_partials(const Geo& g);
// x *= sqrt(E0 / (scale * e2[slot])) for every batch entry (e2 from launch_inner)
void launch_scale_energy(const Geo& g, double2* x, double E0, double scale, const double* e2, cudaStream_t s);

}  // namespace pnop
