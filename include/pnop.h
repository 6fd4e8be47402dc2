/*
 * pnop — forward and adjoint time steps of the perturbation Navier–Stokes
 * equations in a periodic pipe around a Sexl–Womersley base flow, and the
 * checkpointed adjoint sweep that returns the gradient of the final
 * perturbation energy with respect to the initial perturbation
 * (Keuchel & Avila, "Nonlinear optimal perturbation growth in pulsatile pipe
 * flow": Section 2, Eq. 2.1–2.12 for the equations, Section 2.4 for the
 * discretisation and the predictor–corrector step, Section 2.5 and
 * Eq. 2.18–2.21 for the binomial and two-level checkpointing), with the
 * adjoint-looping optimisation of Section 2.3 and the continuous adjoint
 * equations Eq. 2.9–2.11 on top.
 *
 * C ABI, one CUDA device, plain pointers.  Every entry point returns an int
 * status (PNOP_OK = 0, negative on error) unless stated otherwise; no
 * exception crosses the ABI.  The text of the last error of a context is
 * returned by pnop_last_error().
 *
 * Field layout (all field pointers): complex128, interleaved (re, im),
 * C order [3][nr][2M+1][K+1]:
 *   component c = 0,1,2  ->  u_r, u_theta, u_z
 *   radial index j       ->  r_j, j = 0 is the wall r = 1, r decreasing
 *   azimuthal index      ->  m = -M .. M
 *   axial index          ->  k = 0 .. K, wavenumber kz = 2 pi k / Lz
 * f(r,theta,z) = sum_{k=-K..K} sum_{m=-M..M} fhat_{m,k}(r) e^{i(m theta + kz z)}
 * with fhat_{-m,-k} = conj(fhat_{m,k}) (Eq. 2.16); only k >= 0 is stored, so
 * the k = 0 plane must satisfy fhat_{-m,0} = conj(fhat_{m,0}).
 *
 * Ownership: callers own every field buffer they pass; the library never
 * frees them and keeps no pointer to them after a call returns.  The context
 * owns its operators, workspace and checkpoint pool (device memory).
 *
 * Streams: the device work of a call is ordered after earlier work on the
 * stream given to pnop_create (NULL = legacy default stream) and before later
 * work on it; inside a call the context also runs work on its own side and
 * copy streams, forked from and joined back to that stream with events.
 * Calls that return host scalars (energy, inner, gradient) synchronise that
 * stream.  A context must not be used from two host threads at once.
 */
#ifndef PNOP_H
#define PNOP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PNOP_OK = 0,
    PNOP_ERR_INVALID_ARG = -1,  /* bad size, NULL pointer, unsupported combination */
    PNOP_ERR_OOM = -2,          /* device allocation failed or HBM budget exceeded */
    PNOP_ERR_CUDA = -3,         /* a CUDA runtime call or kernel launch failed */
    PNOP_ERR_NONFINITE = -4,    /* a NaN/Inf energy was produced */
    PNOP_ERR_TIMEOUT = -5,      /* device work did not complete within the host limit */
    PNOP_ERR_UNSUPPORTED = -6   /* grid/solver combination not supported */
};

/* Arithmetic of a context, two independent bits:
 *   PNOP_MIXED (1): the theta/z transforms and the products u x w (and their
 *     transposes) in FP32;
 *   PNOP_DF (2): the explicit banded radial products (curl, divergence,
 *     pressure gradient and their transposes) in double-FP32 arithmetic
 *     (about 48 significant bits, Dekker 1971), since FP64 runs at 1/64 of
 *     the FP32 rate on this GPU.
 * Everything else (the radial banded solves, the influence and flux
 * corrections, the base flow, the stage combinations, energies and inner
 * products) stays FP64.  PNOP_FP64 (0) is FP64 throughout. */
enum { PNOP_FP64 = 0, PNOP_MIXED = 1, PNOP_DF = 2, PNOP_MIXED_DF = 3 };

/* Grid.  nr radial points (>= 9); ntheta, nz nominal azimuthal/axial sizes,
 * giving |m| <= M = ntheta/2 - 1 and 0 <= k <= K = nz/2 - 1; the physical
 * (3/2-dealiased) grid is 3(M+1) x 3(K+1) and both must factor into 2s and
 * 3s.  Lz is the pipe length in radii; stretch in [0,1) blends the Chebyshev
 * radial points with uniform spacing (Section 2.4, "relaxation"; 0 = pure
 * Chebyshev). */
typedef struct {
    int nr, ntheta, nz;
    double Lz, stretch;
} pnop_grid;

/* Physics and run parameters.  Re = D Ubar / nu (mean), Wo and A as in
 * Section 1 (Eq. 2.4); time unit R/(2 Ubar), so the pulsation period is
 * 2 pi Re / Wo^2.  dt is the fixed time step, tau0 the start time of the
 * perturbation.  precision: PNOP_FP64, PNOP_MIXED, PNOP_DF or PNOP_MIXED_DF
 * (see above).  snap_budget: checkpoint slots for
 * pnop_gradient including the initial state (>= 1; Section 2.5).
 * snap_budget <= 0 sizes the checkpoint pool from the HBM budget.
 * hbm_budget: bytes the context may allocate (0 = no limit). */
typedef struct {
    double Re, Wo, A, dt, tau0;
    int precision;
    int snap_budget;
    size_t hbm_budget;
} pnop_params;

typedef struct pnop_ctx pnop_ctx;

/* Build the grid, the finite-difference and banded-LU operators, the
 * influence and flux vectors (Section 2.4) and the workspace on the current
 * device.  cuda_stream is a cudaStream_t (may be NULL).  On success *out
 * receives a new context; on failure *out is NULL and the status says why
 * (use pnop_error_string for the text). */
int pnop_create(const pnop_grid* grid, const pnop_params* params, void* cuda_stream, pnop_ctx** out);

/* Replace Re, Wo, A and tau0 (Eq. 2.3–2.4).  Rebuilds the Re-dependent
 * operators when Re changes. */
int pnop_set_base_flow(pnop_ctx* ctx, double Re, double Wo, double A, double tau0);

/* Sizes of a context: nr, M, K; any pointer may be NULL. */
int pnop_dims(const pnop_ctx* ctx, int* nr, int* M, int* K);

/* Radial points r_j (host array of nr doubles, j = 0 at the wall). */
int pnop_grid_points(const pnop_ctx* ctx, double* r_out);

/* Advance the device field u (in/out, layout above) by nsteps predictor-
 * corrector steps (Section 2.4) starting at time t. */
int pnop_step_forward(pnop_ctx* ctx, void* u, double t, int nsteps);

/* One adjoint step: lam (device, in/out) <- J^+ lam, where J is the
 * Jacobian of the forward step taken from the device state u_n at time t_n,
 * and J^+ its adjoint in the energy inner product of Eq. 2.2 (so that
 * <J v, lam> = <v, J^+ lam> for all v).  This is the exact transpose of the
 * discrete step, the discrete counterpart of Eq. 2.9–2.11. */
int pnop_step_adjoint(pnop_ctx* ctx, const void* u_n, void* lam, double t_n);

/* Gradient of E(tau0 + horizon) with respect to the initial perturbation
 * (Eq. 2.8 and 2.12 without the energy multiplier; the paper's u_dagger at
 * tau0 is the negative of grad_out).  u0 (device, read only) is first scaled
 * to energy E0 when E0 > 0, else used as given.  The forward sweep stores
 * snap_budget checkpoints on the binomial schedule of Eq. 2.18–2.20 and the
 * backward sweep recomputes the missing states.  grad_out (device) receives
 * the Riesz representer of dE(T)/du0 in the energy inner product; gain_out
 * (host, may be NULL) receives G = E(T)/E(tau0) (Eq. 2.1).  horizon must be
 * a whole number of time steps (to 1e-9 relative). */
int pnop_gradient(pnop_ctx* ctx, const void* u0, double E0, double horizon, void* grad_out, double* gain_out);

/* Gradient from the continuous adjoint equations (Eq. 2.9-2.11), the form the
 * paper integrates: the same checkpointed forward sweep, then w = -u_dagger
 * from w(T) = u(T) (Eq. 2.8) backward to tau0 with the predictor-corrector of
 * the forward step and the adjoint forcing (PNOP_OP_NONLINEAR_ADJ), taken at
 * the stored forward states of both ends of each step.  grad_out receives
 * w(tau0), the gradient in the energy inner product; it approximates the exact
 * discrete gradient of pnop_gradient to discretisation error.  Other
 * arguments as pnop_gradient.  Allocates on first use physical scratch for 18
 * fields and four more device fields (counted against hbm_budget; not in
 * pnop_context_bytes). */
int pnop_gradient_continuous(pnop_ctx* ctx, const void* u0, double E0, double horizon, void* grad_out,
                             double* gain_out);

/* pnop_gradient in two halves, for reverse-mode drivers (an autograd
 * backward): pnop_gradient_forward copies u0 (rescaled to E0 when E0 > 0),
 * runs the checkpointed forward sweep up to the terminal state u_N and
 * returns E(T) in *ET_out (and the initial energy in *E0_out, may be NULL);
 * the checkpoints stay in the context.  pnop_gradient_backward then runs the
 * reverse sweep with terminal cotangent gE * dE/du_N and writes
 * gE * dE(T)/du0 to grad_out: the Riesz representer in the energy inner
 * product when euclidean = 0, or the Euclidean cotangent of the stored real
 * and imaginary parts (d/dRe + i d/dIm) when euclidean != 0.  Any other call
 * on the context in between (steps, operators, another gradient) discards
 * the pending sweep; pnop_gradient_backward then returns
 * PNOP_ERR_INVALID_ARG.  With snap_budget <= 0 the number of checkpoint slots
 * is as many as fit in hbm_budget (or 80% of free device memory), at most the
 * number of steps (store-all). */
int pnop_gradient_forward(pnop_ctx* ctx, const void* u0, double E0, double horizon, double* ET_out, double* E0_out);
int pnop_gradient_backward(pnop_ctx* ctx, double gE, int euclidean, void* grad_out);

/* Same as pnop_gradient with host buffers: u0_host and grad_host are host
 * arrays in the field layout; the copies are part of the call. */
int pnop_gradient_host(pnop_ctx* ctx, const double* u0_host, double E0, double horizon, double* grad_host,
                       double* gain_out);

/* Counts of the last pnop_gradient: forward steps executed outside the
 * adjoint steps (recomputation included), adjoint steps, checkpoint stores.
 * Any pointer may be NULL. */
int pnop_gradient_stats(const pnop_ctx* ctx, long long* advances, long long* adjoint_steps, long long* stores);

/* Second checkpoint level in pinned host memory (the file level of the
 * two-level schedule, Section 2.5, with Grace memory over the host link in
 * place of disc).  With max_host_slots > 0, each later gradient sweep of N
 * steps with s HBM slots picks the number nf <= max_host_slots of host
 * checkpoints that minimises the recovery time of Eq. 2.21,
 *   nf * T_io + (forward steps) * T_step,
 * counting the forward steps of the schedule exactly (forward phase to the
 * last of nf + 1 near-equal intervals, then each interval's binomial schedule,
 * Eq. 2.18); nf = 0 keeps the single-level schedule.  io_ratio = T_io/T_step
 * for one store plus one load of a field; io_ratio < 0 measures it now on
 * this device.  Host slots (one field each, pinned) are allocated on demand
 * and kept until pnop_destroy; their copies run on a copy stream and overlap
 * the steps (the next load is prefetched).  The gradient is bitwise the same
 * with or without the host level.  max_host_slots = 0 turns the level off.
 * Errors: PNOP_ERR_INVALID_ARG for negative or absurd slot counts,
 * PNOP_ERR_OOM when pinned host memory cannot be allocated. */
int pnop_set_host_tier(pnop_ctx* ctx, long long max_host_slots, double io_ratio);

/* Host level of the last gradient sweep: host checkpoints used, host stores
 * and loads, and the io_ratio in force.  Any pointer may be NULL. */
int pnop_host_tier_stats(const pnop_ctx* ctx, int* host_checkpoints, long long* host_stores, long long* host_loads,
                         double* io_ratio);

/* Host only: the schedule pnop_set_host_tier would choose for nsteps steps
 * with snaps HBM slots, at most max_host_slots host checkpoints and the given
 * io_ratio (>= 0): host checkpoints in *host_checkpoints and forward steps of
 * the sweep (terminal step included) in *advances. */
int pnop_two_level_counts(long long nsteps, int snaps, long long max_host_slots, double io_ratio,
                          int* host_checkpoints, long long* advances);

/* Energy of every Fourier mode of the device field u (Eq. 2.1 weights),
 * split into the cross-section part (u_r, u_theta) in spectrum[0][m + M][k]
 * and the axial part (u_z) in spectrum[1][m + M][k]; spectrum is a host array
 * of 2 (2M+1)(K+1) doubles and sums to pnop_energy(u).  Sections 2.4 and 3 use
 * it: the resolution measures e_M, e_K (the energy of |m| = M, respectively
 * k = K, over 2 E0), the component growths G_z, G_(r,theta), and per-mode
 * energy traces. */
int pnop_mode_energy(pnop_ctx* ctx, const void* u, double* spectrum);

/* Resolution measures of Section 2.4, reduced on the device from the field u
 * (device, layout above): *e_M = the energy of the highest azimuthal mode
 * m = M summed over the full axial spectrum k = -K..K, and *e_K = the energy
 * of the highest axial mode k = K summed over m = -M..M, each over E0 (the
 * paper keeps both below 1e-8 when it chooses M and K).  The printed formulas
 * are garbled (their prefactors and the summation index of e_K); this reads
 * them as energy fractions of those mode shells, with the energy of Eq. 2.1.
 * The full-spectrum energies follow from the stored half by the Hermitian
 * symmetry f(-m, -k) = conj f(m, k).  E0 <= 0 takes the energy of u itself.
 * Host outputs; the call synchronises the context's stream.  Single-request
 * contexts only.  Errors: PNOP_ERR_INVALID_ARG for NULL pointers or a
 * non-finite E0, PNOP_ERR_NONFINITE when the result is not finite. */
int pnop_resolution(pnop_ctx* ctx, const void* u, double E0, double* e_M, double* e_K);

/* Counters and result of pnop_optimise. */
typedef struct {
    int iterations;    /* accepted updates */
    int gradients;     /* reverse sweeps (one per accepted point, the start included) */
    int forward_evals; /* forward sweeps of the line search (the start included) */
    int converged;     /* 1 when R < tol ended the loop, or the gradient is parallel to u0 */
    double gain;       /* G = E(T)/E0 of the returned u0 */
    double rel_change; /* last R = |G^(s+1) - G^s| / G^(s+1) */
} pnop_opt_stats;

/* Adjoint-looping optimisation of the initial perturbation (Section 2.3):
 * u0 (device, in/out) is projected onto admissible fields (PNOP_OP_PROJECT)
 * and scaled to energy E0, then repeatedly replaced by
 * (1 + lambda alpha) u0 - alpha u_dagger with u_dagger = -P grad (the paper's
 * adjoint field at tau0; grad as returned by pnop_gradient, projected so that
 * the iterates stay admissible), lambda the root lambda_+ of the energy
 * constraint (Eq. 2.14) and alpha found by backtracking: alpha_max of
 * Eq. 2.15 first, halved while the gain G does not grow.  A trial whose sweep
 * is not finite counts as a step that did not raise G.  The loop ends when an
 * accepted update changes G by a relative R < tol (the paper uses 1e-8), when
 * the line search cannot raise G before R drops below tol, when the gradient
 * is parallel to u0 (to rounding), or after max_iter accepted updates.  u0
 * holds the last accepted perturbation.  gain_history (host, may be NULL)
 * receives max_iter + 1 doubles: G of the start and after each accepted
 * update (entries beyond stats->iterations are left unchanged).  stats (host)
 * may be NULL.  Each trial point costs one checkpointed forward sweep;
 * accepted points add the reverse sweep.  Uses two more device fields of the
 * context and the projection factors on first call.  The loop keeps no state
 * between calls besides u0: calling again with the returned u0 resumes it
 * (the first iterate is then the last accepted one). */
int pnop_optimise(pnop_ctx* ctx, void* u0, double E0, double horizon, int max_iter, double tol,
                  double* gain_history, pnop_opt_stats* stats);

/* pnop_optimise with the choice of adjoint: PNOP_ADJOINT_DISCRETE (the exact
 * gradient of pnop_gradient, the default of pnop_optimise) or
 * PNOP_ADJOINT_CONTINUOUS (the paper's continuous adjoint equations, as in
 * pnop_gradient_continuous). */
enum { PNOP_ADJOINT_DISCRETE = 0, PNOP_ADJOINT_CONTINUOUS = 1 };
int pnop_optimise_ex(pnop_ctx* ctx, void* u0, double E0, double horizon, int max_iter, double tol, int adjoint,
                     double* gain_history, pnop_opt_stats* stats);

/* First trial step of every line search of pnop_optimise and
 * pnop_optimise_ex, as a fraction of alpha_max: 0 < alpha_frac <= 1, with 1
 * (the default) the paper's choice.  At alpha = alpha_max the discriminant of
 * the scaling lambda (Eq. 2.14) is zero, and its square root amplifies the
 * rounding of the update, so two implementations agree on the iterates only
 * to about the square root of their gradients' agreement; a fraction below 1
 * keeps the update well conditioned, which lets a caller compare iterates at
 * full precision.  PNOP_ERR_INVALID_ARG for a null context or a fraction
 * outside (0, 1]. */
int pnop_set_optimiser_first_step(pnop_ctx* ctx, double alpha_frac);

/* Operators of the step, applied to device fields (for testing and for
 * users who compose their own schemes; layout as above, all FP64 in/out):
 *   PNOP_OP_CURL       out = curl a                              (Eq. 2.5)
 *   PNOP_OP_NONLINEAR  out = N(a, t) = a x w + (U e_z) x w + a x (-U' e_theta),
 *                      w = curl a, products on the 3/2-padded grid
 *   PNOP_OP_STAGE      out = S(a, b): one predictor-corrector stage with
 *                      velocity a and forcing b (pressure projection, Crank-
 *                      Nicolson Helmholtz solves, influence and flux
 *                      corrections; Section 2.4)
 *   PNOP_OP_NONLINEAR_T out = (dN/da at a, t)^T b
 *   PNOP_OP_STAGE_T_U  out = (dS/da)^T a      (b unused)
 *   PNOP_OP_STAGE_T_F  out = (dS/db)^T a      (b unused)
 *   PNOP_OP_NONLINEAR_ADJ out = N_adj(b; a, t): forcing of the continuous adjoint
 *                      equation for the adjoint field b (w = -u_dagger) about the
 *                      forward state a, in backward time (Eq. 2.9):
 *                      U db/dz - b_z U' e_r + P[-a x curl b - 2 (grad a) . b]
 *   PNOP_OP_PROJECT    out = P a: orthogonal projection, in the energy inner
 *                      product, onto admissible fields (Hermitian k = 0 plane,
 *                      zero at the wall, discrete divergence zero at every
 *                      r_j, mean mode with u_r = 0 and zero flux; the
 *                      constraints of Section 2.2)  (b unused)
 * Transposes act on Euclidean cotangents of the stored real and imaginary
 * parts.  out must not alias a or b. */
enum {
    PNOP_OP_CURL = 0,
    PNOP_OP_NONLINEAR = 1,
    PNOP_OP_STAGE = 2,
    PNOP_OP_NONLINEAR_T = 3,
    PNOP_OP_STAGE_T_U = 4,
    PNOP_OP_STAGE_T_F = 5,
    PNOP_OP_PROJECT = 6,
    PNOP_OP_NONLINEAR_ADJ = 7
};
int pnop_apply(pnop_ctx* ctx, int op, const void* a, const void* b, void* out, double t);

/* Host limit (seconds, 0 = none) on every wait of the context for its device
 * work.  When a wait passes the limit the call returns PNOP_ERR_TIMEOUT; the
 * queued work is not aborted and keeps running on the device, and the
 * context stays usable: pnop_sync (or any later synchronising call) waits
 * for it.  Results of the timed-out call are undefined. */
int pnop_set_timeout(pnop_ctx* ctx, double seconds);

/* Waits (without limit) for all device work of the context. */
int pnop_sync(pnop_ctx* ctx);

/* Kernel classes for launch counting and device timing. */
enum {
    PNOP_K_SYNTH_THETA = 0,  /* zero-padded inverse theta FFTs (units: FFT columns) */
    PNOP_K_ZPASS_FWD = 1,    /* z FFTs + u x w products (units: (j, theta) rows) */
    PNOP_K_ZPASS_ADJ = 2,    /* z FFTs + transposed products (units: rows) */
    PNOP_K_ANAL_THETA = 3,   /* forward theta FFTs + truncation (units: FFT columns) */
    PNOP_K_SPECTRAL = 4,     /* curl, base-flow terms and their transposes (units: algorithmic FP64 flops) */
    PNOP_K_RADIAL_BAND = 5,  /* banded radial matvecs, +/- basis, influence (units: algorithmic FP64 flops) */
    PNOP_K_RADIAL_SOLVE = 6, /* banded LU solves (units: systems of nr unknowns) */
    PNOP_K_ELEMENTWISE = 7,  /* axpby, energy weights (units: values) */
    PNOP_K_REDUCE = 8,       /* inner-product reductions (units: values) */
    PNOP_K_NCLASS = 9
};

/* Start counting (and, for the classes set in class_mask, timing with CUDA
 * events on the context stream around each launch); resets the counters.
 * class_mask = 0 counts launches without timing. */
int pnop_profile(pnop_ctx* ctx, unsigned class_mask);

/* Measured fused-multiply-add throughput of the current device, in TFLOP/s
 * (2 flops per FMA): precision PNOP_FP64 times FP64 FMAs, PNOP_MIXED FP32
 * FMAs.  This is the denominator of the ALU roofline of the library's
 * FP64-bound kernels (the paper gives no performance figures; this is a
 * measurement utility).  Every SM runs independent FMA chains for about
 * `seconds` (0 < seconds <= 10) per launch, in nine configurations (4, 8 or
 * 16 chains per thread, 2, 4 or 8 blocks of 256 threads per SM), three
 * launches each; the best rate is returned in *tflops (host).  The work is ordered on cuda_stream (NULL =
 * legacy default stream) and the call synchronises it.  No device memory is
 * allocated.  Bad arguments return PNOP_ERR_INVALID_ARG, CUDA failures
 * PNOP_ERR_CUDA. */
int pnop_measure_fma_peak(int precision, double seconds, void* cuda_stream, double* tflops);

/* Read the counters since pnop_profile: per class device milliseconds (timed
 * classes only), kernel launches and work units (arrays of PNOP_K_NCLASS;
 * any may be NULL).  Synchronises the stream. */
int pnop_profile_read(pnop_ctx* ctx, double* ms, long long* launches, double* units);

/* E = (1/2) <u, u> (Eq. 2.1–2.2) of a device field; written to *E_out. */
int pnop_energy(pnop_ctx* ctx, const void* u, double* E_out);

/* <a, b> = int int int a . b r dr dtheta dz (Eq. 2.2) of two device fields. */
int pnop_inner(pnop_ctx* ctx, const void* a, const void* b, double* out);

/* Device bytes a context of this grid and precision allocates with `snaps`
 * checkpoint slots (an upper estimate, for admission control by an HBM
 * budget).  Host only; needs no device. */
int pnop_context_bytes(const pnop_grid* grid, const pnop_params* params, int snaps, size_t* bytes);

/* Device bytes the context holds right now (operators, workspace, checkpoint
 * slots, host-tier staging; buffers allocated on first use are included once
 * they exist).  The checkpoint pool grows to the largest slot count a sweep
 * has used and is kept until pnop_destroy, so this is the memory cost of the
 * snapshot budget of Section 2.5 as run.  Host only: reads a counter, issues
 * no device work.  NULL arguments return PNOP_ERR_INVALID_ARG. */
int pnop_device_bytes(const pnop_ctx* ctx, size_t* bytes);

/* Binomial checkpoint plan (Section 2.5) for nsteps steps and snaps slots,
 * computed on the host: minimal forward recomputations (Eq. 2.18), stores.
 * Needs no device. */
int pnop_revolve_counts(int nsteps, int snaps, long long* advances, long long* stores);

/* Energy without any device allocation (the paper has no counterpart; this
 * is a library convenience).  For callers that cannot call cudaMalloc where
 * they need the result: code running after all device memory has been handed
 * to another allocator or a fixed pool (a new cudaMalloc would fail there),
 * or loops that must not call cudaMalloc/cudaFree because those can
 * synchronise the device and stall other streams.  Such callers cannot create
 * a context, so none is needed: pass the field u (device, layout above, nr,
 * M, K as for a context), the radial quadrature weights W (device, nr
 * doubles: sum_j W_j f(r_j) = int_0^1 f r dr, the same radial quadrature as
 * the context's inner product uses) and the pipe length Lz; *E_out (host)
 * receives (1/2) <u, u>, as pnop_energy would.  The work is ordered on
 * cuda_stream (NULL = legacy default stream) and the call synchronises it.
 *
 * Scratch: a fixed array in device global memory inside the library (32 KiB
 * of partial sums plus one result slot); every GPU that loads the library
 * holds it until the process exits.  The first call on a device resolves that
 * array's device address (with the device current) and should therefore come
 * before any stream capture on that device.  All calls share the array:
 * calls whose device work overlaps (concurrent streams or host threads)
 * race on it and must be serialised by the caller.  Each call writes every
 * part of the array it reads before reading it, so nothing a previous call left
 * there reaches the result.  The cached address is only valid while the
 * device's primary context lives: do not call cudaDeviceReset between calls.
 *
 * Limits and errors: 3 * nr * (2M+1) * (K+1) may be at most
 * PNOP_NOALLOC_MAX_VALUES complex values; larger fields, NULL pointers or bad
 * sizes return PNOP_ERR_INVALID_ARG before any device work; CUDA failures
 * return PNOP_ERR_CUDA, a NaN/Inf energy PNOP_ERR_NONFINITE. */
#define PNOP_NOALLOC_MAX_VALUES (16777216LL) /* 2^24 complex values (268 MB field) */
int pnop_energy_noalloc(const void* u, const double* W, int nr, int M, int K, double Lz, double* E_out,
                        void* cuda_stream);

/* Error text of the last failing call on ctx ("" when none). */
const char* pnop_last_error(const pnop_ctx* ctx);

/* Static text for a status code. */
const char* pnop_error_string(int status);

/* Free the context and everything it owns.  NULL is allowed. */
void pnop_destroy(pnop_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched gradients (a serving form; the paper has no counterpart).  A batch
 * holds up to `capacity` (1..PNOP_MAX_BATCH) gradient requests of one grid,
 * each with its own Re, Wo, A, dt, tau0, E0 and horizon, and runs them
 * together: every kernel of a forward or adjoint step is launched once for
 * all requests that take that kind of step next (the requests' fields sit in
 * per-request slots of shared buffers).  Each request follows its own
 * binomial checkpoint schedule (Section 2.5, snap_budget slots of its own)
 * and gets bitwise the gradient and gain pnop_gradient returns for it on a
 * single context with the same snap_budget and precision.  Requests can be
 * submitted while others run (continuous batching).
 *
 * Use: pnop_batch_create; pnop_batch_submit per request (copies u0 in, the
 * slot is taken until its result is fetched); pnop_batch_run to queue steps;
 * pnop_batch_poll to see whether a request is finished without blocking;
 * pnop_batch_result to fetch its gradient (same semantics as pnop_gradient's
 * grad_out) and gain and free its slot.  All device work is ordered on the
 * stream given at creation; submit, run and poll do not wait for the device,
 * result waits for the request's own work. */
#define PNOP_MAX_BATCH 16
typedef struct pnop_batch pnop_batch;

/* grid: as for pnop_create.  params: precision, snap_budget (>= 1,
 * checkpoint slots per request) and hbm_budget (0 = no limit) apply to every
 * request; Re, Wo, A, dt and tau0 must be valid but are replaced by each
 * request's own.  Device memory for all slots is allocated here (about
 * capacity times a single context's workspace plus snap_budget fields). */
int pnop_batch_create(const pnop_grid* grid, const pnop_params* params, int capacity, void* cuda_stream,
                      pnop_batch** out);

/* Admit one request: physics from request->Re, Wo, A, dt, tau0 (the other
 * fields are ignored), u0 (device, layout above, read during the call's
 * stream-ordered copy), E0 > 0 rescales u0 to energy E0 (E0 <= 0 keeps it),
 * horizon a positive whole number of steps of request->dt.  *id_out receives
 * the request id.  PNOP_ERR_OOM when no slot is free, PNOP_ERR_INVALID_ARG
 * for bad parameters; builds the request's operators on the host. */
int pnop_batch_submit(pnop_batch* batch, const pnop_params* request, const void* u0, double E0, double horizon,
                      int* id_out);

/* The host part of a submission, split off so that it can run beside the
 * device work: pnop_batch_prepare builds the operators of one request's
 * physics (Re, Wo, A, dt, tau0 of *request) on the host.  It reads only the
 * batch's grid tables, which never change after creation, records no error
 * text, and may run on any number of host threads at once, concurrently with
 * every other call on the batch.  pnop_batch_submit_prepared then admits a
 * request with them (same arguments and errors as pnop_batch_submit; ops
 * stays owned by the caller and may be used again); pnop_ops_free releases
 * them (NULL allowed).  pnop_batch_submit is prepare + submit_prepared. */
typedef struct pnop_ops pnop_ops;
int pnop_batch_prepare(const pnop_batch* batch, const pnop_params* request, pnop_ops** out);
int pnop_batch_submit_prepared(pnop_batch* batch, const pnop_ops* ops, const void* u0, double E0, double horizon,
                               int* id_out);
void pnop_ops_free(pnop_ops* ops);

/* Queue up to max_ticks batched steps (one tick: every request's pending
 * checkpoint copies, then one batched forward, terminal or adjoint step for
 * the requests whose next step is of the most common kind).  *ticks_out:
 * ticks queued (fewer when all requests are finished); *running_out:
 * requests still unfinished after them.  Either pointer may be NULL. */
int pnop_batch_run(pnop_batch* batch, int max_ticks, int* ticks_out, int* running_out);

/* *done_out = 1 when request id has been fully queued and its device work
 * has completed, else 0.  PNOP_ERR_INVALID_ARG for an unknown id. */
int pnop_batch_poll(pnop_batch* batch, int id, int* done_out);

/* Gradient (device, may be NULL) and gain of a finished request; frees its
 * slot.  PNOP_ERR_INVALID_ARG when the request has not been fully queued
 * yet (run more ticks), PNOP_ERR_NONFINITE when its energies are not finite
 * (the slot is freed all the same). */
int pnop_batch_result(pnop_batch* batch, int id, void* grad_out, double* gain_out);

/* Batched steps launched (ticks), the requests they covered in total
 * (entries / ticks = mean batch size) and the kernels launched. */
int pnop_batch_stats(const pnop_batch* batch, long long* ticks, long long* entries, long long* launches);

/* Device bytes pnop_batch_create allocates for this grid, precision
 * (params->precision), checkpoint slots (params->snap_budget) and capacity (an
 * upper estimate, for admission control by an HBM budget).  Host only; needs
 * no device. */
int pnop_batch_bytes(const pnop_grid* grid, const pnop_params* params, int capacity, size_t* bytes);

const char* pnop_batch_last_error(const pnop_batch* batch);
void pnop_batch_destroy(pnop_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* PNOP_H */
