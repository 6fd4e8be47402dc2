// C ABI of the GB300 pipe-flow forward/adjoint solver: context set-up, the
// predictor-corrector step (Section 2.4), its exact transpose, and the
// binomially checkpointed gradient sweep (Section 2.5, Eq. 2.18-2.20).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <complex>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/pnop.h"
#include "kernels.hpp"
#include "setup.hpp"

static_assert(pnop::kSK == pnop::kTileK, "solver block and factor tile must cover the same k");

using pnop::Geo;

namespace {

struct CudaError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
struct Status : std::runtime_error {
    int code;
    Status(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

// NVTX range over a scope (step, stage, sweep), for timeline tools and for
// ncu --nvtx filters; a no-op when no tool is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Binomial schedule (Section 2.5) as a list of actions: advance n steps from
// the state in a slot (into another slot, or into the scratch state when dst
// is -1), or take the adjoint step of step n from a slot / the scratch state.
// One entry of a checkpointing plan.  kAdv: advance n steps from snapshot
// `slot` (result into snapshot `dst`, or left as the current state when
// dst < 0); kAdj: the adjoint step `start` from snapshot `slot` (or the
// current state); kStore / kLoad: copy snapshot `slot` to / from host slot
// `host` (the second level of the two-level schedule).
enum ActionKind { kAdv = 0, kAdj = 1, kStore = 2, kLoad = 3 };
struct Action {
    int kind;
    long long start, n;
    int slot, dst, host;
};

// One request of a batched context, as a queue of per-slot operations: copies
// between the slot's state and its checkpoints, forward steps, the terminal
// step, adjoint steps and the final Riesz map.
enum OpKind { kOpRestore = 0, kOpStore = 1, kOpFwd = 2, kOpTerm = 3, kOpAdj = 4, kOpFinish = 5 };
struct Op {
    int kind;
    long long n;  // step index (kOpFwd, kOpTerm, kOpAdj)
    int snap;     // checkpoint index (kOpRestore, kOpStore)
};
struct BatchReq {
    bool active = false, done = false, fetched = true;
    int id = -1;
    double Re = 0, Wo = 0, A = 0, dt = 0, tau0 = 0, omega = 0, E0 = 0;
    long long N = 0;
    std::vector<Op> ops;
    size_t pos = 0;
    cudaEvent_t ev_done = nullptr;
};

bool smooth_size(int n) {
    if (n < 2) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

}  // namespace

struct pnop_ctx {
    pnop::HostOps h;
    pnop_params prm{};
    cudaStream_t stream = nullptr;
    Geo geo{};
    size_t bytes = 0;
    std::vector<void*> allocs;
    // operators
    double *d_r = nullptr, *d_invr = nullptr, *d_W = nullptr, *d_D1 = nullptr, *d_Lb = nullptr;
    double *d_facH = nullptr, *d_facP = nullptr, *d_infl = nullptr, *d_fluxg = nullptr;
    double *d_facHT = nullptr, *d_facPT = nullptr;
    double* d_projL = nullptr;  // admissible-projection factors, built on first use
    double* d_dgt = nullptr;    // 1/dt - k_z^2/(2 Re) per k (depends on dt and Re)
    double* d_spec = nullptr;   // per-mode energies [2][nm][nk]
    double2 *d_Uh = nullptr, *d_dUh = nullptr;
    pnop::Twiddles tw{};
    // workspace
    double2* omega = nullptr;
    double2* N0 = nullptr;  // also second F-bar of the adjoint step
    double2* N1 = nullptr;
    double2* us = nullptr;
    double2* ua = nullptr;
    double2* Fb = nullptr;
    double2* Nb = nullptr;
    double2* ubs = nullptr;
    double2* wb = nullptr;
    double2* R = nullptr;
    double2* Rl = nullptr;  // front part of the transposed stage for the incoming cotangent
    double2* ac = nullptr;  // per-mode coefficients of the transposed influence correction [slot][m][k]
    double* pw = nullptr;   // wall partials of the forward Helmholtz solve [slot][3][m][k] complex
    double2* q = nullptr;
    double2* q2 = nullptr;  // pressure scratch of the side stream
    cudaStream_t side = nullptr;  // second stream for independent work within a step
    cudaEvent_t ev_fork = nullptr, ev_t = nullptr, ev_base = nullptr;
    double2* Nbase = nullptr;  // base-flow terms (or their transpose), added by the analysis
    double2 *tmpA = nullptr, *tmpB = nullptr, *lamA = nullptr, *lamB = nullptr;
    void* Y = nullptr;
    void* Y2 = nullptr;  // theta synthesis of u and curl u kept from N(u) for N'(u)^T in the adjoint step
    void* Z = nullptr;
    double* partial = nullptr;
    double* dscal = nullptr;  // [4] device scalars
    std::vector<double2*> snaps;
    std::string err;
    long long st_adv = 0, st_adj = 0, st_store = 0;
    // gradient sweep state (schedule, position, scratch state, terminal state)
    std::vector<Action> plan;
    size_t plan_pos = 0;
    const double2* cur = nullptr;
    double2* uN = nullptr;
    double2 *opt_g = nullptr, *opt_u = nullptr;  // adjoint looping: gradient, trial point
    // continuous adjoint (allocated on first use): physical scratch for 18 fields,
    // grad u (9 component planes), the later forward state u^{n+1}
    void* Y3 = nullptr;
    double2 *Gu = nullptr, *cprev = nullptr;
    bool continuous = false;  // run_plan takes the continuous adjoint step
    // second checkpoint level in pinned host memory (two-level schedule)
    long long host_max = 0;            // host slots allowed (0: single level)
    double host_ratio = 0;             // T_io / T_step of Eq. 2.21 (store + load of one field)
    std::vector<void*> host;           // pinned host slots, allocated on demand
    double2* hstage = nullptr;         // device staging field for the copies
    cudaStream_t copy = nullptr;       // copy stream (host traffic overlaps the steps)
    cudaEvent_t ev_copy = nullptr, ev_staged = nullptr;
    int pref_host = -1;                // host slot prefetched into hstage (-1: none)
    int st_nf = 0;
    long long st_hstore = 0, st_hload = 0;
    bool pending = false;
    int st_slots = 0;
    double timeout_s = 0;  // host limit on waits for device work (0: none)
    double opt_alpha_frac = 1.0;  // first line-search step of the optimiser, in units of alpha_max
    // recomputation beside the adjoint: a second workspace on its own streams
    // that runs the reverse sweep's forward advances while the adjoint steps
    // run on this context's stream (single-request contexts, discrete adjoint,
    // single checkpoint level)
    pnop_ctx* shadow = nullptr;
    double2* ring[2] = {nullptr, nullptr};       // end states of advances to the scratch state
    cudaEvent_t ev_ring_w[2] = {}, ev_ring_r[2] = {};  // ring buffer written (shadow) / last read (adjoint)
    std::vector<cudaEvent_t> ev_slot_w, ev_slot_r;     // per checkpoint slot, created on first use
    std::vector<char> slot_shadow;                     // slot written by the shadow in this sweep
    cudaEvent_t ev_main = nullptr, ev_shadow = nullptr;
    bool owns_stream = false;                          // the shadow created its stream
    // per-class launch counters, work units and optional event timing
    unsigned prof_mask = 0;
    std::vector<cudaEvent_t> ev;     // pairs (start, stop)
    std::vector<int> ev_cls;         // class of each recorded pair
    size_t ev_used = 0;
    double prof_ms[PNOP_K_NCLASS] = {};
    long long launches[PNOP_K_NCLASS] = {};
    double units[PNOP_K_NCLASS] = {};
    // batched context: nslot storage slots, one request each; every spectral
    // buffer (fields, checkpoints, scratch) holds nslot fields at stride 3 S
    int nslot = 1;
    bool batched = false;
    double bt[pnop::kMaxBatch] = {};  // step start time of each entry of the current batched launch
    std::vector<BatchReq> breq;       // per slot
    int next_id = 0;
    double2* bcur = nullptr;          // per-slot current state
    double2* blam = nullptr;          // per-slot cotangent
    double *d_e0 = nullptr, *d_eT = nullptr;  // per-slot 2 E(0) and 2 E(T) (inner products)
    long long b_ticks = 0, b_launch_entries = 0;

    size_t S() const { return (size_t)h.d.nr * h.d.nm * h.d.nk; }
    size_t field_bytes() const { return 3 * S() * sizeof(double2); }

    void* dalloc(size_t n) {
        if (prm.hbm_budget && bytes + n > prm.hbm_budget)
            throw Status(PNOP_ERR_OOM, "HBM budget exceeded (" + std::to_string(bytes + n) + " > " +
                                           std::to_string(prm.hbm_budget) + " bytes)");
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Status(PNOP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        allocs.push_back(p);
        bytes += n;
        return p;
    }
    template <class T> T* upload(const std::vector<T>& v) {
        T* p = (T*)dalloc(std::max<size_t>(1, v.size()) * sizeof(T));
        if (!v.empty()) ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
        return p;
    }
    double2* field() { return (double2*)dalloc((size_t)nslot * field_bytes()); }
};

namespace {

std::vector<double2> cvec(const std::vector<std::complex<double>>& v) {
    std::vector<double2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = make_double2(v[i].real(), v[i].imag());
    return o;
}

// (hi, lo) float pairs of FP64 values: hi the nearest float, lo the nearest
// float to the remainder (tables of the double-FP32 kernels)
float2 split_pair(double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
std::vector<float2> split_pairs(const std::vector<double>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = split_pair(v[i]);
    return o;
}

template <class T2> std::vector<T2> twiddle_table(int N) {
    std::vector<T2> t(N);
    for (int n = 0; n < N; ++n) {
        long double a = -2.0L * 3.14159265358979323846264338327950288L * n / N;
        t[n].x = (decltype(t[n].x))std::cos(a);
        t[n].y = (decltype(t[n].y))std::sin(a);
    }
    return t;
}

// Tables of slot `slot` from the operators h was built with (Re, dt, Wo and
// A of that slot's request).  The per-slot tables are allocated for all slots
// on first use; the grid-only tables (pressure factors) are written once.
void upload_slot_operators(pnop_ctx* c, int slot, const pnop::HostOps& h) {
    const size_t ns = (size_t)c->nslot;
    auto put = [&](double*& dst, const std::vector<double>& v, size_t slots, size_t at) {
        if (!dst) dst = (double*)c->dalloc(std::max<size_t>(1, v.size()) * slots * sizeof(double));
        ck(cudaMemcpy(dst + at * v.size(), v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice), "upload");
    };
    {
        // device bands hold L_m / (2 Re): the explicit Crank-Nicolson half B = 1/dt + L/(2 Re)
        std::vector<double> lb(h.Lb);
        for (double& x : lb) x /= 2.0 * h.ph.Re;
        put(c->d_Lb, lb, ns, slot);
        c->geo.sLb = lb.size();
    }
    {
        std::vector<double> dg(h.d.nk);
        for (int k = 0; k < h.d.nk; ++k) {
            const double kz = 2.0 * M_PI * k / h.d.Lz;
            dg[k] = 1.0 / h.ph.dt - kz * kz / (2.0 * h.ph.Re);
        }
        put(c->d_dgt, dg, ns, slot);
        c->geo.sNk = dg.size();
    }
    put(c->d_facH, h.facH, ns, slot);
    put(c->d_facHT, h.facHT, ns, slot);
    c->geo.sFacH = h.facH.size();
    if (!c->d_facP) {
        put(c->d_facP, h.facP, 1, 0);
        put(c->d_facPT, h.facPT, 1, 0);
    }
    put(c->d_infl, h.infl, ns, slot);
    c->geo.sInfl = h.infl.size();
    put(c->d_fluxg, h.fluxg, ns, slot);
    c->geo.sNr = h.fluxg.size();
    auto uh = cvec(h.Uh), duh = cvec(h.dUh);
    if (!c->d_Uh) {
        c->d_Uh = (double2*)c->dalloc(uh.size() * ns * sizeof(double2));
        c->d_dUh = (double2*)c->dalloc(duh.size() * ns * sizeof(double2));
    }
    ck(cudaMemcpy(c->d_Uh + slot * uh.size(), uh.data(), uh.size() * sizeof(double2), cudaMemcpyHostToDevice), "upload");
    ck(cudaMemcpy(c->d_dUh + slot * duh.size(), duh.data(), duh.size() * sizeof(double2), cudaMemcpyHostToDevice),
       "upload");
    Geo& g = c->geo;
    g.two_dt[slot] = 2.0 / h.ph.dt;
    g.two_dtf[slot] = split_pair(2.0 / h.ph.dt);
    g.flux_inv[slot] = h.flux_inv;
    g.Lb = c->d_Lb;
    g.dgt = c->d_dgt;
    g.facH = c->d_facH;
    g.facP = c->d_facP;
    g.facHT = c->d_facHT;
    g.facPT = c->d_facPT;
    g.ntile = h.ntile;
    g.infl = c->d_infl;
    g.fluxg = c->d_fluxg;
    g.Uh = c->d_Uh;
    g.dUh = c->d_dUh;
}

// operator tables that depend on Re/dt/Wo/A are re-uploaded on change
void upload_operators(pnop_ctx* c) { upload_slot_operators(c, 0, c->h); }

bool mixed(const pnop_ctx* c) { return (c->prm.precision & PNOP_MIXED) != 0; }

void prof_flush(pnop_ctx* c) {
    if (!c->ev_used) return;
    ck(cudaEventSynchronize(c->ev[2 * c->ev_used - 1]), "profile sync");
    for (size_t i = 0; i < c->ev_used; ++i) {
        float ms = 0;
        ck(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]), "profile elapsed");
        c->prof_ms[c->ev_cls[i]] += ms;
    }
    c->ev_used = 0;
}

// Launch `nk` kernels of class `cls` doing `units` work units per batch entry
// on stream `st` (the context stream by default); bracket them with CUDA
// events on that stream when the class is being timed.
template <class F> void run(pnop_ctx* c, int cls, int nk, double units, F&& f, cudaStream_t st) {
    c->launches[cls] += nk;
    c->units[cls] += units * c->geo.nb;
    if (!(c->prof_mask & (1u << cls))) {
        f();
        return;
    }
    const size_t pool = 8192;
    if (c->ev.empty()) {
        c->ev.resize(2 * pool);
        c->ev_cls.resize(pool);
        for (auto& e : c->ev) ck(cudaEventCreate(&e), "event create");
    }
    if (c->ev_used == pool) prof_flush(c);
    ck(cudaEventRecord(c->ev[2 * c->ev_used], st), "event record");
    f();
    ck(cudaEventRecord(c->ev[2 * c->ev_used + 1], st), "event record");
    c->ev_cls[c->ev_used++] = cls;
}
template <class F> void run(pnop_ctx* c, int cls, int nk, double units, F&& f) {
    run(c, cls, nk, units, std::forward<F>(f), c->stream);
}

// Fork: work queued on the side stream after this call starts after all work
// queued so far on the context stream.
void fork_side(pnop_ctx* c) {
    ck(cudaEventRecord(c->ev_fork, c->stream), "fork");
    ck(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork");
}
// Join: work queued on the context stream after this call waits for `e`,
// recorded on the side stream.
void join_side(pnop_ctx* c, cudaEvent_t e) { ck(cudaStreamWaitEvent(c->stream, e, 0), "join"); }

double nmodes(const pnop_ctx* c) { return (double)c->h.d.nm * c->h.d.nk; }

// Waits for the context stream.  With a timeout set, polls the stream until
// the deadline and then gives up with PNOP_ERR_TIMEOUT: the queued work keeps
// running and a later call (or pnop_sync) waits for it; nothing is aborted.
void wait_stream(pnop_ctx* c, const char* what) {
    if (!(c->timeout_s > 0)) {
        ck(cudaStreamSynchronize(c->stream), what);
        return;
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return;
        if (e != cudaErrorNotReady) ck(e, what);
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > c->timeout_s)
            throw Status(PNOP_ERR_TIMEOUT, std::string(what) + ": device work not finished within the host limit");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Algorithmic FP64 flops per value of the banded/spectral kernels (work units
// of the RADIAL_BAND and SPECTRAL classes): a 9-entry band row on a complex
// value is 36 flops; the remaining terms are counted as written.
namespace flops {
constexpr double div = 36 + 12, rhs = 36 + 12 + 8, rhs_u = 6 + 12, a0_mode = 72, finish = 20, finish_u = 6;
constexpr double tfinish = 36, trhs_u = 12 + 12, trhs_f = 8, qbar = 36 + 8, tdiv = 36 + 12;
constexpr double curl = 2 * 36 + 16, curlT = 2 * 36 + 20, base = 12, grad_u = 3 * 36 + 24;
}  // namespace flops

// out = [addto +] S(u, F), one predictor-corrector stage (Section 2.4); u
// null: forcing only, S(0, F).  The old velocity enters the Helmholtz
// right-hand side as (2/dt) T u and is subtracted after the solve, which
// equals the explicit Crank-Nicolson half B u because A + B = 2 I / dt.
void stage(pnop_ctx* c, const double2* u, const double2* F, double2* out, const double2* addto) {
    Range nvtx_range("pnop:stage");
    const Geo& g = c->geo;
    cudaStream_t s = c->stream;
    const double S = (double)c->S();
    run(c, PNOP_K_RADIAL_BAND, 1, flops::div * S, [&] { pnop::launch_stage_div(g, F, c->q, s); });
    run(c, PNOP_K_RADIAL_SOLVE, 1, nmodes(c), [&] { pnop::launch_stage_psolve(g, c->q, s); });
    run(c, PNOP_K_RADIAL_BAND, 1, (flops::rhs + (u ? flops::rhs_u : 0)) * S,
        [&] { pnop::launch_stage_rhs(g, u, F, c->q, c->R, s); });
    run(c, PNOP_K_RADIAL_SOLVE, 1, 3 * nmodes(c), [&] { pnop::launch_stage_hsolve(g, c->R, u, c->pw, s); });
    run(c, PNOP_K_RADIAL_BAND, 1, (flops::finish + (u ? flops::finish_u : 0)) * S + flops::a0_mode * nmodes(c),
        [&] { pnop::launch_stage_finish(g, c->R, addto, u, c->pw, out, s); });
}

// out = S(u, F) on the context stream alone (operator access)
void stage_u(pnop_ctx* c, const double2* u, const double2* F, double2* out) { stage(c, u, F, out, nullptr); }

// Rb = A^{-T} Ti^H Fin^H ubn [+ add]: the part of the transposed stage shared
// by its velocity and forcing cotangents.  The per-mode coefficients of
// Fin^H go to c->ac (added to what it holds when ac_add), for the velocity
// part of stageT_rhs.
void stageT_front(pnop_ctx* c, const double2* ubn, double2* Rb, cudaStream_t s, const double2* add = nullptr,
                  int ac_add = 0) {
    const Geo& g = c->geo;
    run(c, PNOP_K_RADIAL_BAND, 1, flops::tfinish * c->S(),
        [&] { pnop::launch_stageT_finish(g, ubn, Rb, c->ac, ac_add, s); }, s);
    run(c, PNOP_K_RADIAL_SOLVE, 1, 3 * nmodes(c), [&] { pnop::launch_stageT_hsolve(g, Rb, add, s); }, s);
}

// Fb <- Proj^H Fb (transposed pressure projection, in place, scratch q)
void stageT_proj(pnop_ctx* c, double2* Fb, double2* q, cudaStream_t s) {
    const Geo& g = c->geo;
    const double S = (double)c->S();
    run(c, PNOP_K_RADIAL_BAND, 1, flops::qbar * S, [&] { pnop::launch_stageT_qbar(g, Fb, q, s); }, s);
    run(c, PNOP_K_RADIAL_SOLVE, 1, nmodes(c), [&] { pnop::launch_stageT_psolve(g, q, s); }, s);
    run(c, PNOP_K_RADIAL_BAND, 1, flops::tdiv * S, [&] { pnop::launch_stageT_div(g, q, Fb, s); }, s);
}

// ub (=, or += when acc) S_u^H ubn ; Fb = S_F^H ubn  (either may be null)
void stageT(pnop_ctx* c, const double2* ubn, double2* ub, int acc, double2* Fb) {
    Range nvtx_range("pnop:stageT");
    const Geo& g = c->geo;
    stageT_front(c, ubn, c->R, c->stream);
    run(c, PNOP_K_RADIAL_BAND, 1, ((ub ? flops::trhs_u : 0) + (Fb ? flops::trhs_f : 0)) * c->S(),
        [&] { pnop::launch_stageT_rhs(g, c->R, nullptr, 1.0, 0.0, ub, acc, Fb, ubn, nullptr, c->ac, c->stream); });
    if (Fb) stageT_proj(c, Fb, c->q, c->stream);
}

// u <- P u, the energy-orthogonal projection onto admissible fields (scratch q)
void project(pnop_ctx* c, double2* u) {
    if (!c->d_projL) {
        std::vector<double> L;
        std::string err;
        if (!pnop::build_projection(c->h, L, err)) throw Status(PNOP_ERR_UNSUPPORTED, err);
        c->d_projL = c->upload(L);
    }
    run(c, PNOP_K_RADIAL_SOLVE, 4, nmodes(c), [&] { pnop::launch_project(c->geo, u, c->q, c->d_projL, c->stream); });
}

void axpby(pnop_ctx* c, double a, const double2* x, double b, const double2* y, double2* out) {
    const size_t n = 3 * c->S();
    run(c, PNOP_K_ELEMENTWISE, 1, (double)n, [&] { pnop::launch_axpby(c->geo, n, a, x, b, y, out, c->stream); });
}
void weight(pnop_ctx* c, const double2* x, double2* out, int divide) {
    run(c, PNOP_K_ELEMENTWISE, 1, 3.0 * c->S(), [&] { pnop::launch_weight(c->geo, x, out, divide, c->stream); });
}
void inner_dev(pnop_ctx* c, const double2* a, const double2* b, double* dst) {
    run(c, PNOP_K_REDUCE, 2, 3.0 * c->S(), [&] { pnop::launch_inner(c->geo, a, b, c->partial, dst, c->stream); });
}

// theta synthesis / z pass / theta analysis in the context's transform
// precision, through the physical scratch Y.  Fields [0, cached) are already
// synthesised in Y and are not redone.
void transforms(pnop_ctx* c, const pnop::FieldPtrs& f, int nin, int nout, int zmode, const pnop::ZScales& sc, void* Y,
                int cached, cudaEvent_t before_analysis) {
    const Geo& g = c->geo;
    cudaStream_t s = c->stream;
    const double cols = (double)g.nr * g.nk, rows = (double)g.nr * g.nt;
    const int zk = zmode == pnop::ZFWD ? PNOP_K_ZPASS_FWD : PNOP_K_ZPASS_ADJ;
    pnop::FieldPtrs fs = f;
    for (int i = 0; i + cached < nin; ++i) {
        fs.in[i] = f.in[cached + i];
        fs.inf[i] = f.inf[cached + i];
    }
    const int ns = nin - cached;
    const size_t plane = (size_t)g.nr * g.nt * g.nk;
    if (mixed(c)) {
        float2* Yf = (float2*)Y;
        run(c, PNOP_K_SYNTH_THETA, 1, ns * cols, [&] { pnop::launch_synth_theta<float2>(g, fs, ns, Yf + cached * plane, c->tw, s); });
        run(c, zk, 1, rows, [&] { pnop::launch_zpass<float2>(g, zmode, Yf, (float2*)c->Z, sc, c->tw, s); });
        if (before_analysis) join_side(c, before_analysis);
        run(c, PNOP_K_ANAL_THETA, 1, nout * cols, [&] { pnop::launch_anal_theta<float2>(g, f, nout, (const float2*)c->Z, c->tw, s); });
    } else {
        double2* Yd = (double2*)Y;
        run(c, PNOP_K_SYNTH_THETA, 1, ns * cols, [&] { pnop::launch_synth_theta<double2>(g, fs, ns, Yd + cached * plane, c->tw, s); });
        run(c, zk, 1, rows, [&] { pnop::launch_zpass<double2>(g, zmode, Yd, (double2*)c->Z, sc, c->tw, s); });
        if (before_analysis) join_side(c, before_analysis);
        run(c, PNOP_K_ANAL_THETA, 1, nout * cols, [&] { pnop::launch_anal_theta<double2>(g, f, nout, (const double2*)c->Z, c->tw, s); });
    }
}

// ------------------------------------------------------------------ nonlinear term
// Pulsation phase (cos, sin of omega t) of every batch entry into geo.cs
// for the next launches.  A single-request context takes t itself; a batched
// context reads t as a step offset (0: the entry's step start, 1: its end)
// and adds it to the entry's own start time with its own dt and omega.
void set_phase(pnop_ctx* c, double t) {
    Geo& g = c->geo;
    if (!c->batched) {
        const double ph = c->h.omega * t;
        g.cs[0] = make_double2(std::cos(ph), std::sin(ph));
        return;
    }
    for (int b = 0; b < g.nb; ++b) {
        const BatchReq& r = c->breq[g.slot[b]];
        const double ph = r.omega * (c->bt[b] + t * r.dt);
        g.cs[b] = make_double2(std::cos(ph), std::sin(ph));
    }
}

// Base-flow terms of N(u) at time t into Nbase on the side stream (the caller
// has forked it); the analysis of the transforms adds them after ev_base.
void queue_base(pnop_ctx* c, const double2* u, double t) {
    set_phase(c, t);
    run(c, PNOP_K_SPECTRAL, 1, flops::base * c->S(), [&] { pnop::launch_base(c->geo, u, c->Nbase, c->side); },
        c->side);
    ck(cudaEventRecord(c->ev_base, c->side), "record");
}

// w = curl u into the context's vorticity buffer, which becomes transform
// inputs first_w..first_w+2, and u itself inputs first_u..first_u+2.  When
// the transforms run in FP32 (the vorticity's only reader, which takes it
// rounded to FP32 anyway), w is stored in FP32 and the curl also writes u
// rounded to FP32, so that the synthesis reads both without converting; in
// FP64 u is read where it is.  The buffer holds nslot slots of 3 S double2,
// i.e. 6 S nslot float2; the kernels offset an FP32 field of slot s by
// s * 3 S values, so w takes the first 3 S nslot float2 and u the rest.
void curl_into(pnop_ctx* c, const double2* u, pnop::FieldPtrs& f, int first_w, int first_u) {
    const Geo& g = c->geo;
    const size_t S = c->S();
    cudaStream_t s = c->stream;
    if (mixed(c)) {
        float2* w = reinterpret_cast<float2*>(c->omega);
        float2* uf = w + (size_t)c->nslot * 3 * S;
        run(c, PNOP_K_SPECTRAL, 1, flops::curl * S, [&] { pnop::launch_curl_f32(g, u, w, uf, s); });
        for (int i = 0; i < 3; ++i) {
            f.inf[first_w + i] = w + i * S;
            f.inf[first_u + i] = uf + i * S;
        }
    } else {
        run(c, PNOP_K_SPECTRAL, 1, flops::curl * S, [&] { pnop::launch_curl(g, u, c->omega, s); });
        for (int i = 0; i < 3; ++i) {
            f.in[first_w + i] = c->omega + i * S;
            f.in[first_u + i] = u + i * S;
        }
    }
}

// N = P[I(u) x I(w)] - U du/dz - u_r dU/dr e_z, w = curl u  (Eq. 2.5; base-flow
// terms in advective form, computed on the side stream while the curl and the
// transforms run).  The physical u and w are left in Y (fields 0..5).  With
// base_queued the caller has already queued the base terms of this u.
void nonlinear(pnop_ctx* c, const double2* u, double t, double2* N, void* Y, bool base_queued = false) {
    Range nvtx_range("pnop:nonlinear");
    const Geo& g = c->geo;
    const size_t S = c->S();
    cudaStream_t s = c->stream;
    if (!base_queued) {
        fork_side(c);
        queue_base(c, u, t);
    }
    pnop::FieldPtrs f{};
    curl_into(c, u, f, 3, 0);
    for (int i = 0; i < 3; ++i) {
        f.out[i] = N + i * S;
        f.add[i] = c->Nbase + i * S;
    }
    pnop::ZScales sc{};
    const double inv_n = 1.0 / ((double)g.nt * g.nzp);
    for (int i = 0; i < 6; ++i) sc.h0[i] = sc.hk[i] = 1.0;
    for (int i = 0; i < 3; ++i) sc.o0[i] = sc.ok[i] = inv_n;
    transforms(c, f, 6, 3, pnop::ZFWD, sc, Y, 0, c->ev_base);
}

// ub = (dN/du at u)^T nb  (Euclidean cotangents).  With cached, Y already
// holds the physical u and curl u of this u (fields 0..5, left by nonlinear).
// The base-flow transpose runs on the side stream and is added by the analysis.
void nonlinearT(pnop_ctx* c, const double2* u, double t, const double2* nb, double2* ub, void* Y, bool cached) {
    Range nvtx_range("pnop:nonlinearT");
    const Geo& g = c->geo;
    const size_t S = c->S();
    cudaStream_t s = c->stream;
    fork_side(c);
    set_phase(c, t);
    run(c, PNOP_K_SPECTRAL, 1, flops::base * S, [&] { pnop::launch_baseT(g, nb, c->Nbase, c->side); }, c->side);
    ck(cudaEventRecord(c->ev_base, c->side), "record");
    pnop::FieldPtrs f{};
    if (!cached) curl_into(c, u, f, 3, 0);
    // the vorticity cotangent is a pure FP32 product in the mixed path (no
    // FP64 term is added to it): the analysis writes it in FP32
    float2* wbf = mixed(c) ? reinterpret_cast<float2*>(c->wb) : nullptr;
    for (int i = 0; i < 3; ++i) {
        f.in[6 + i] = nb + i * S;
        f.out[i] = ub + i * S;
        if (wbf) f.outf[3 + i] = wbf + i * S;
        else f.out[3 + i] = c->wb + i * S;
        f.add[i] = c->Nbase + i * S;
    }
    pnop::ZScales sc{};
    const double inv_n = 1.0 / ((double)g.nt * g.nzp);
    for (int i = 0; i < 6; ++i) sc.h0[i] = sc.hk[i] = 1.0;
    // transpose of the truncated analysis: (1/N) sum_k Re(nb e^{i phi}), no c_k
    for (int i = 6; i < 9; ++i) {
        sc.h0[i] = inv_n;
        sc.hk[i] = 0.5 * inv_n;
    }
    // transpose of the synthesis: c_k sum g e^{-i phi}
    for (int i = 0; i < 6; ++i) {
        sc.o0[i] = 1.0;
        sc.ok[i] = 2.0;
    }
    transforms(c, f, 9, 6, pnop::ZADJ, sc, Y, cached ? 6 : 0, c->ev_base);
    run(c, PNOP_K_SPECTRAL, 1, flops::curlT * S, [&] {
        if (wbf) pnop::launch_curlT_acc_f32(g, wbf, ub, s);
        else pnop::launch_curlT_acc(g, c->wb, ub, s);
    });
}

// ------------------------------------------------------------------ continuous adjoint
// Forcing of the adjoint equation in backward time (Eq. 2.9, with w = -u_dagger):
// N_adj(w; u, t) = U dw/dz - w_z dU/dr e_r + P[-u x curl w - 2 (grad u) . w];
// the base-flow part on the side stream (queued by the caller when
// base_queued), added by the analysis.
void queue_base_adj(pnop_ctx* c, const double2* w, double t) {
    set_phase(c, t);
    run(c, PNOP_K_SPECTRAL, 1, flops::base * c->S(), [&] { pnop::launch_base_adj(c->geo, w, c->Nbase, c->side); },
        c->side);
    ck(cudaEventRecord(c->ev_base, c->side), "record");
}

void nonlinear_adj(pnop_ctx* c, const double2* w, const double2* u, double t, double2* N, bool base_queued = false) {
    Range nvtx_range("pnop:nonlinear_adj");
    const Geo& g = c->geo;
    const size_t S = c->S();
    cudaStream_t s = c->stream;
    if (!c->Y3) {
        const size_t cz = mixed(c) ? sizeof(float2) : sizeof(double2);
        c->Y3 = c->dalloc(18 * (size_t)g.nr * g.nt * g.nk * cz);
    }
    if (!c->Gu) c->Gu = (double2*)c->dalloc(9 * S * sizeof(double2));
    if (!base_queued) {
        fork_side(c);
        queue_base_adj(c, w, t);
    }
    pnop::FieldPtrs f{};
    curl_into(c, w, f, 3, 6);
    run(c, PNOP_K_SPECTRAL, 1, flops::grad_u * S, [&] { pnop::launch_grad_u(g, u, c->Gu, s); });
    for (int i = 0; i < 3; ++i) {
        f.in[i] = u + i * S;
        f.out[i] = N + i * S;
        f.add[i] = c->Nbase + i * S;
    }
    for (int i = 0; i < 9; ++i) f.in[9 + i] = c->Gu + i * S;
    pnop::ZScales sc{};
    const double inv_n = 1.0 / ((double)g.nt * g.nzp);
    for (int i = 0; i < 18; ++i) sc.h0[i] = sc.hk[i] = 1.0;
    for (int i = 0; i < 3; ++i) sc.o0[i] = sc.ok[i] = inv_n;
    transforms(c, f, 18, 3, pnop::ZCADJ, sc, c->Y3, 0, c->ev_base);
}

// w(t_now) from w(t_next = t_now + dt): the predictor-corrector of the forward
// step run backward in time, forcing N_adj at (u_next, t_next) for the
// predictor and at (u_now, t_now) for the corrector; S is the same stage map.
void cadj_step(pnop_ctx* c, const double2* u_next, double t_next, const double2* u_now, double t_now,
               const double2* w, double2* out) {
    Range nvtx_range("pnop:cadj_step");
    fork_side(c);
    queue_base_adj(c, w, t_next);
    nonlinear_adj(c, w, u_next, t_next, c->N0, true);
    stage(c, w, c->N0, c->us, nullptr);
    nonlinear_adj(c, c->us, u_now, t_now, c->N1);
    axpby(c, 0.5, c->N1, -0.5, c->N0, c->N1);
    stage(c, nullptr, c->N1, out, c->us);
}

// ------------------------------------------------------------------ steps
// Predictor u* = S(u, N0), corrector S(u, (N0 + N*)/2) = u* + S(0, (N* - N0)/2)
// (S is linear), so the corrector has no velocity part.
void fwd_step(pnop_ctx* c, const double2* u, double2* out, double t) {
    Range nvtx_range("pnop:fwd_step");
    fork_side(c);
    queue_base(c, u, t);
    nonlinear(c, u, t, c->N0, c->Y, true);
    stage(c, u, c->N0, c->us, nullptr);
    nonlinear(c, c->us, t + c->h.ph.dt, c->N1, c->Y);
    axpby(c, 0.5, c->N1, -0.5, c->N0, c->N1);
    stage(c, nullptr, c->N1, out, c->us);
}

// lout = J^T lin (Euclidean cotangents) for the step from state u at time t.
// With u' = S_u u + S_F (N0 + N*)/2, u* = S_u u + S_F N0, N* = N(u*), N0 = N(u):
//   Fb = S_F^H lin, ub* = N*'^T (Fb/2),
//   ubar = S_u^H (lin + ub*) + N0'^T S_F^H (lin/2 + ub*).
// S_u^H and S_F^H share their front part (Rl for lin, R for ub*), so the
// velocity part of the transposed stage runs once, on lin + ub* (the second
// solve adds Rl, the second front adds its Fin^H coefficients to lin's).
// Everything that depends on lin alone (Rl, S_F^H lin) runs on the side
// stream while the predictor is re-run on the context stream.  N(u) and
// N'(u)^T share the physical u and curl u (scratch Y2).
void adj_step(pnop_ctx* c, const double2* u, double t, const double2* lin, double2* lout) {
    Range nvtx_range("pnop:adj_step");
    const Geo& g = c->geo;
    fork_side(c);
    queue_base(c, u, t);
    stageT_front(c, lin, c->Rl, c->side);
    run(c, PNOP_K_RADIAL_BAND, 1, flops::trhs_f * c->S(),
        [&] { pnop::launch_stageT_rhs(g, c->Rl, nullptr, 0.5, 0.0, nullptr, 0, c->Nb, nullptr, nullptr, nullptr,
                                      c->side); },
        c->side);
    stageT_proj(c, c->Nb, c->q2, c->side);  // Nb = S_F^H lin / 2
    ck(cudaEventRecord(c->ev_t, c->side), "record");
    nonlinear(c, u, t, c->N0, c->Y2, true);  // physical u, curl u stay in Y2 for N'(u)^T below
    stage(c, u, c->N0, c->us, nullptr);
    join_side(c, c->ev_t);
    nonlinearT(c, c->us, t + c->h.ph.dt, c->Nb, c->ubs, c->Y, false);
    stageT_front(c, c->ubs, c->R, c->stream, c->Rl, 1);  // R = front(ub*) + front(lin)
    run(c, PNOP_K_RADIAL_BAND, 1, (flops::trhs_u + flops::trhs_f) * c->S(),
        [&] { pnop::launch_stageT_rhs(g, c->R, c->Rl, 1.0, -0.5, c->ua, 0, c->Nb, lin, c->ubs, c->ac, c->stream); });
    stageT_proj(c, c->Nb, c->q, c->stream);  // Nb = S_F^H (lin/2 + ub*)
    nonlinearT(c, u, t, c->Nb, c->ubs, c->Y2, true);
    axpby(c, 1.0, c->ua, 1.0, c->ubs, lout);
}

double inner_sync(pnop_ctx* c, const double2* a, const double2* b) {
    inner_dev(c, a, b, c->dscal);
    double v = 0;
    ck(cudaMemcpyAsync(&v, c->dscal, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "inner copy");
    wait_stream(c, "inner sync");
    return v;
}

// ------------------------------------------------------------------ checkpointed sweep
const double2* advance(pnop_ctx* c, const double2* src, long long start, long long n, double2* dst_final) {
    const double2* cur = src;
    for (long long i = 0; i < n; ++i) {
        double2* out = (i == n - 1 && dst_final) ? dst_final : (cur == c->tmpA ? c->tmpB : c->tmpA);
        fwd_step(c, cur, out, c->h.ph.tau0 + (start + i) * c->h.ph.dt);
        ++c->st_adv;
        cur = out;
    }
    return cur;
}

// Reverse steps [start, start+l) whose first state sits in snapshot `slot`,
// with s slots available (that one included).
void plan_reverse(std::vector<Action>& P, long long start, long long l, int slot, int s) {
    if (l <= 0) return;
    if (l == 1) {
        P.push_back({kAdj, start, 1, slot, 0, -1});
        return;
    }
    if (s == 1) {
        for (long long i = l - 1; i >= 0; --i) {
            if (i > 0) P.push_back({kAdv, start, i, slot, -1, -1});
            P.push_back({kAdj, start + i, 1, i > 0 ? -1 : slot, 0, -1});
        }
        return;
    }
    const int r = pnop::revolve_repetitions(l, s);
    long long m = std::max<long long>(1, std::max(pnop::binom_beta(s, r - 2), l - pnop::binom_beta(s - 1, r)));
    m = std::min(m, l - 1);
    P.push_back({kAdv, start, m, slot, slot + 1, -1});
    plan_reverse(P, start + m, l - m, slot + 1, s - 1);
    plan_reverse(P, start, m, slot, s);
}

// Two-level schedule (Section 2.5): nf >= 1 host checkpoints hold the starts
// b_0 = 0, ..., b_{nf-1} of the first nf of nf + 1 near-equal intervals
// (b_i = floor(i N / (nf + 1))); the last interval starts in snapshot 0.  The
// forward phase stores u0, advances interval by interval storing each start,
// then runs the binomial schedule of the last interval; the reverse phase
// loads each earlier start from the host and runs that interval's schedule.
long long interval_start(long long N, int nf, int i) { return (long long)((__int128)i * N / (nf + 1)); }

void plan_two_level(std::vector<Action>& P, long long N, int s, int nf) {
    P.push_back({kStore, 0, 0, 0, -1, 0});
    for (int i = 1; i <= nf; ++i) {
        const long long b0 = interval_start(N, nf, i - 1), b1 = interval_start(N, nf, i);
        P.push_back({kAdv, b0, b1 - b0, 0, 0, -1});
        if (i < nf) P.push_back({kStore, b1, 0, 0, -1, i});
    }
    const long long bl = interval_start(N, nf, nf);
    plan_reverse(P, bl, N - bl, 0, s);
    for (int i = nf - 1; i >= 0; --i) {
        const long long b0 = interval_start(N, nf, i), b1 = interval_start(N, nf, i + 1);
        P.push_back({kLoad, b0, 0, 0, -1, i});
        plan_reverse(P, b0, b1 - b0, 0, s);
    }
}

// Forward steps of the whole sweep (the terminal step included) with nf host
// checkpoints: the forward phase to the last interval, then each interval's
// binomial recomputation (Eq. 2.18); nf = 0 is the single-level schedule.
double two_level_steps(long long N, int s, int nf) {
    if (nf == 0) return (double)pnop::revolve_advances(N, s) + 1.0;
    const long long L = N / (nf + 1), q = N % (nf + 1);  // q intervals of L + 1, the rest of L
    const double inner = (double)(nf + 1 - q) * (double)pnop::revolve_advances(L, s) +
                         (double)q * (double)pnop::revolve_advances(L + 1, s);
    return (double)interval_start(N, nf, nf) + inner + 1.0;
}

// Number of host checkpoints minimising the recovery time of Eq. 2.21,
// nf T_io + (forward steps) T_step, in units of T_step (ratio = T_io / T_step).
int choose_host_checkpoints(long long N, int s, long long host_max, double ratio) {
    const long long kmax = std::min<long long>(host_max, N - 1);
    int best = 0;
    double best_cost = two_level_steps(N, s, 0);
    for (long long k = 1; k <= kmax; ++k) {
        const double cost = (double)k * ratio + two_level_steps(N, s, (int)k);
        if (cost < best_cost) {
            best_cost = cost;
            best = (int)k;
        }
    }
    return best;
}

// Runs actions [from, to) of the plan; returns the index of the first adjoint
// action reached when stop_at_adjoint (its state pointer in *state).
// ---- second checkpoint level: pinned host memory over the host link
// The staging field hstage carries every host copy; ev_staged marks the last
// context-stream use of it, ev_copy the last copy-stream transfer.
void ensure_host_tier(pnop_ctx* c, int slots) {
    if (!c->copy) {
        ck(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking), "copy stream");
        ck(cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming), "event");
        ck(cudaEventCreateWithFlags(&c->ev_staged, cudaEventDisableTiming), "event");
        ck(cudaEventRecord(c->ev_copy, c->copy), "event");
        ck(cudaEventRecord(c->ev_staged, c->stream), "event");
    }
    if (!c->hstage) c->hstage = c->field();
    while ((int)c->host.size() < slots) {
        void* p = nullptr;
        cudaError_t e = cudaMallocHost(&p, c->field_bytes());
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Status(PNOP_ERR_OOM, std::string("pinned host slot: ") + cudaGetErrorString(e));
        }
        c->host.push_back(p);
    }
}

void host_store(pnop_ctx* c, const double2* src, int h) {
    const size_t fb = c->field_bytes();
    ck(cudaStreamWaitEvent(c->stream, c->ev_copy, 0), "wait copy");  // hstage free
    ck(cudaMemcpyAsync(c->hstage, src, fb, cudaMemcpyDeviceToDevice, c->stream), "stage");
    ck(cudaEventRecord(c->ev_staged, c->stream), "event");
    ck(cudaStreamWaitEvent(c->copy, c->ev_staged, 0), "wait stage");
    ck(cudaMemcpyAsync(c->host[h], c->hstage, fb, cudaMemcpyDeviceToHost, c->copy), "d2h");
    ck(cudaEventRecord(c->ev_copy, c->copy), "event");
    c->pref_host = -1;
    ++c->st_hstore;
}

void host_prefetch(pnop_ctx* c, int h) {
    ck(cudaStreamWaitEvent(c->copy, c->ev_staged, 0), "wait stage");  // hstage no longer read
    ck(cudaMemcpyAsync(c->hstage, c->host[h], c->field_bytes(), cudaMemcpyHostToDevice, c->copy), "h2d");
    ck(cudaEventRecord(c->ev_copy, c->copy), "event");
    c->pref_host = h;
}

// host slot h -> dst, then start the transfer of the plan's next load
void host_load(pnop_ctx* c, int h, double2* dst, size_t plan_index) {
    if (c->pref_host != h) host_prefetch(c, h);
    ck(cudaStreamWaitEvent(c->stream, c->ev_copy, 0), "wait h2d");
    ck(cudaMemcpyAsync(dst, c->hstage, c->field_bytes(), cudaMemcpyDeviceToDevice, c->stream), "unstage");
    ck(cudaEventRecord(c->ev_staged, c->stream), "event");
    c->pref_host = -1;
    ++c->st_hload;
    for (size_t i = plan_index + 1; i < c->plan.size(); ++i)
        if (c->plan[i].kind == kLoad) {
            host_prefetch(c, c->plan[i].host);
            break;
        }
}

size_t run_plan(pnop_ctx* c, size_t from, bool stop_at_adjoint, const double2** state) {
    const auto& P = c->plan;
    for (size_t i = from; i < P.size(); ++i) {
        const Action& a = P[i];
        if (a.kind == kStore) {
            host_store(c, c->snaps[a.slot], a.host);
            continue;
        }
        if (a.kind == kLoad) {
            host_load(c, a.host, c->snaps[a.slot], i);
            continue;
        }
        if (a.kind == kAdv) {
            const double2* r = advance(c, c->snaps[a.slot], a.start, a.n, a.dst >= 0 ? c->snaps[a.dst] : nullptr);
            if (a.dst >= 0) ++c->st_store;
            else c->cur = r;
            continue;
        }
        const double2* st = a.slot >= 0 ? c->snaps[a.slot] : c->cur;
        if (stop_at_adjoint) {
            *state = st;
            return i;
        }
        const double tn = c->h.ph.tau0 + a.start * c->h.ph.dt;
        if (c->continuous) {
            cadj_step(c, c->cprev, tn + c->h.ph.dt, st, tn, c->lamA, c->lamB);
            ck(cudaMemcpyAsync(c->cprev, st, c->field_bytes(), cudaMemcpyDeviceToDevice, c->stream), "keep state");
        } else {
            adj_step(c, st, tn, c->lamA, c->lamB);
        }
        std::swap(c->lamA, c->lamB);
        ++c->st_adj;
    }
    return P.size();
}

// ---- recomputation beside the adjoint
// The shadow is a second workspace for forward steps: its own work fields,
// physical scratch and streams, the context's operator tables.  It is created
// before the checkpoint pool is sized, so its memory counts against the HBM
// budget like the rest of the context.
void ensure_shadow(pnop_ctx* c) {
    if (c->shadow) return;
    pnop_ctx* sh = new pnop_ctx();
    try {
        sh->prm = c->prm;
        sh->prm.hbm_budget = c->prm.hbm_budget ? (c->prm.hbm_budget > c->bytes ? c->prm.hbm_budget - c->bytes : 1) : 0;
        sh->h.d = c->h.d;
        sh->nslot = 1;
        ck(cudaStreamCreateWithFlags(&sh->stream, cudaStreamNonBlocking), "shadow stream");
        sh->owns_stream = true;
        ck(cudaStreamCreateWithFlags(&sh->side, cudaStreamNonBlocking), "shadow side stream");
        for (cudaEvent_t* e : {&sh->ev_fork, &sh->ev_t, &sh->ev_base})
            ck(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event");
        for (double2** b : {&sh->omega, &sh->N0, &sh->N1, &sh->us, &sh->R, &sh->Nbase, &sh->tmpA, &sh->tmpB})
            *b = sh->field();
        sh->q = (double2*)sh->dalloc(c->S() * sizeof(double2));
        sh->pw = (double*)sh->dalloc((size_t)3 * c->h.d.nm * c->h.d.nk * sizeof(double2));
        const size_t cz = mixed(c) ? sizeof(float2) : sizeof(double2);
        const size_t plane = (size_t)c->h.d.nr * c->h.d.nth * c->h.d.nk * cz;
        sh->Y = sh->dalloc(9 * plane);
        sh->Z = sh->dalloc(6 * plane);
        for (int r = 0; r < 2; ++r) {
            ck(cudaEventCreateWithFlags(&c->ev_ring_w[r], cudaEventDisableTiming), "event");
            ck(cudaEventCreateWithFlags(&c->ev_ring_r[r], cudaEventDisableTiming), "event");
        }
        ck(cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming), "event");
        ck(cudaEventCreateWithFlags(&c->ev_shadow, cudaEventDisableTiming), "event");
    } catch (...) {
        pnop_destroy(sh);
        throw;
    }
    c->shadow = sh;
    c->bytes += sh->bytes;
    c->ring[0] = c->field();
    c->ring[1] = c->field();
}

// The shadow's view of the context as it is now (operators, phase, dt, profiling).
void sync_shadow(pnop_ctx* c) {
    pnop_ctx* sh = c->shadow;
    sh->geo = c->geo;
    sh->tw = c->tw;
    sh->h.ph = c->h.ph;
    sh->h.omega = c->h.omega;
    sh->prm.precision = c->prm.precision;
    sh->prof_mask = c->prof_mask;
}

cudaEvent_t slot_event(std::vector<cudaEvent_t>& v, int slot) {
    if ((int)v.size() <= slot) v.resize(slot + 1, nullptr);
    if (!v[slot]) ck(cudaEventCreateWithFlags(&v[slot], cudaEventDisableTiming), "event");
    return v[slot];
}

// Reverse part of a single-level plan with its forward advances on the
// shadow, so that recomputing the states of the next adjoint steps runs on
// the GPU beside the adjoint steps of the present ones.  Events order every
// buffer: an adjoint step waits for the advance that wrote its state; an
// advance into a checkpoint slot (or one of the two scratch end states)
// waits for the adjoint steps that last read it.  The kernels and their
// inputs are those of run_plan, so the gradient is bitwise the same.
void run_plan_overlap(pnop_ctx* c, size_t from) {
    Range nvtx_range("pnop:reverse_overlap");
    pnop_ctx* sh = c->shadow;
    sync_shadow(c);
    const auto& P = c->plan;
    const size_t ns = c->snaps.size();
    std::vector<char> wrote(ns, 0), read(ns, 0);
    bool ring_read[2] = {false, false};
    int ring_next = 0, cur_ring = -1;
    const double2* cur = c->cur;
    ck(cudaEventRecord(c->ev_main, c->stream), "event");  // the shadow starts after the forward phase
    ck(cudaStreamWaitEvent(sh->stream, c->ev_main, 0), "wait");
    for (size_t i = from; i < P.size(); ++i) {
        const Action& a = P[i];
        if (a.kind == kAdv) {
            double2* dst = nullptr;
            int r = -1;
            if (a.dst >= 0) {
                if (read[a.dst]) ck(cudaStreamWaitEvent(sh->stream, slot_event(c->ev_slot_r, a.dst), 0), "wait");
                dst = c->snaps[a.dst];
            } else {
                r = ring_next;
                ring_next ^= 1;
                if (ring_read[r]) ck(cudaStreamWaitEvent(sh->stream, c->ev_ring_r[r], 0), "wait");
                dst = c->ring[r];
            }
            advance(sh, c->snaps[a.slot], a.start, a.n, dst);
            c->st_adv += a.n;
            if (a.dst >= 0) {
                ck(cudaEventRecord(slot_event(c->ev_slot_w, a.dst), sh->stream), "event");
                wrote[a.dst] = 1;
                ++c->st_store;
            } else {
                ck(cudaEventRecord(c->ev_ring_w[r], sh->stream), "event");
                cur = dst;
                cur_ring = r;
            }
            continue;
        }
        if (a.kind != kAdj) throw Status(PNOP_ERR_INVALID_ARG, "overlapped sweep: host-level action in the plan");
        const double2* st = cur;
        if (a.slot >= 0) {
            st = c->snaps[a.slot];
            if (wrote[a.slot]) ck(cudaStreamWaitEvent(c->stream, slot_event(c->ev_slot_w, a.slot), 0), "wait");
        } else if (cur_ring >= 0) {
            ck(cudaStreamWaitEvent(c->stream, c->ev_ring_w[cur_ring], 0), "wait");
        }
        adj_step(c, st, c->h.ph.tau0 + a.start * c->h.ph.dt, c->lamA, c->lamB);
        std::swap(c->lamA, c->lamB);
        ++c->st_adj;
        if (a.slot >= 0) {
            ck(cudaEventRecord(slot_event(c->ev_slot_r, a.slot), c->stream), "event");
            read[a.slot] = 1;
        } else if (cur_ring >= 0) {
            ck(cudaEventRecord(c->ev_ring_r[cur_ring], c->stream), "event");
            ring_read[cur_ring] = true;
        }
    }
    ck(cudaEventRecord(c->ev_shadow, sh->stream), "event");
    ck(cudaStreamWaitEvent(c->stream, c->ev_shadow, 0), "wait");
    // the shadow's launches belong to this context's counters
    prof_flush(sh);
    for (int k = 0; k < PNOP_K_NCLASS; ++k) {
        c->launches[k] += sh->launches[k];
        c->units[k] += sh->units[k];
        c->prof_ms[k] += sh->prof_ms[k];
        sh->launches[k] = 0;
        sh->units[k] = 0;
        sh->prof_ms[k] = 0;
    }
}

// Count-only replay of the same schedule (host logic, no device work).
void count_reverse(long long l, int s, long long& adv, long long& stores) {
    if (l <= 1) return;
    if (s == 1) {
        adv += l * (l - 1) / 2;
        return;
    }
    const int r = pnop::revolve_repetitions(l, s);
    long long m = std::max<long long>(1, std::max(pnop::binom_beta(s, r - 2), l - pnop::binom_beta(s - 1, r)));
    m = std::min(m, l - 1);
    adv += m;
    ++stores;
    count_reverse(l - m, s - 1, adv, stores);
    count_reverse(m, s, adv, stores);
}

int fail(pnop_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

template <class F> int guarded(pnop_ctx* c, F&& fn) {
    if (!c) return PNOP_ERR_INVALID_ARG;
    c->err.clear();
    try {
        return fn();
    } catch (const Status& s) {
        return fail(c, s.code, s.what());
    } catch (const CudaError& e) {
        return fail(c, PNOP_ERR_CUDA, e.what());
    } catch (const std::runtime_error& e) {
        return fail(c, PNOP_ERR_CUDA, e.what());
    } catch (const std::bad_alloc&) {
        return fail(c, PNOP_ERR_OOM, "host allocation failed");
    }
}

// Number of checkpoint slots: the configured budget, or (budget <= 0) as many
// as fit in the context's HBM budget (or 80% of free device memory), at most N.
int snapshot_slots(pnop_ctx* c, long long N) {
    long long s = c->prm.snap_budget;
    if (s <= 0) {
        size_t avail = 0;
        if (c->prm.hbm_budget) {
            avail = c->prm.hbm_budget > c->bytes ? c->prm.hbm_budget - c->bytes : 0;
        } else {
            size_t fr = 0, tot = 0;
            ck(cudaMemGetInfo(&fr, &tot), "memory info");
            avail = (size_t)(0.8 * (double)fr);
        }
        s = (long long)c->snaps.size() + (long long)(avail / c->field_bytes());
    }
    s = std::max<long long>(1, std::min<long long>(s, N));
    return (int)s;
}

// T_io / T_step of Eq. 2.21 on this device: one store and one load of a field
// through pinned host memory against one forward step, timed with events.
double measure_io_ratio(pnop_ctx* c) {
    ensure_host_tier(c, 1);
    const size_t fb = c->field_bytes();
    struct Events {  // destroyed on every exit path
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        ~Events() {
            for (auto x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    cudaEvent_t* e = ev.e;
    for (int i = 0; i < 3; ++i) ck(cudaEventCreate(&e[i]), "event");
    ck(cudaMemsetAsync(c->tmpB, 0, fb, c->stream), "memset");
    float io = 0, step = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first round warms up
        ck(cudaEventRecord(e[0], c->stream), "event");
        ck(cudaMemcpyAsync(c->host[0], c->tmpB, fb, cudaMemcpyDeviceToHost, c->stream), "d2h");
        ck(cudaMemcpyAsync(c->hstage, c->host[0], fb, cudaMemcpyHostToDevice, c->stream), "h2d");
        ck(cudaEventRecord(e[1], c->stream), "event");
        fwd_step(c, c->tmpB, c->tmpA, c->h.ph.tau0);
        ck(cudaEventRecord(e[2], c->stream), "event");
        ck(cudaEventSynchronize(e[2]), "sync");
        ck(cudaEventElapsedTime(&io, e[0], e[1]), "elapsed");
        ck(cudaEventElapsedTime(&step, e[1], e[2]), "elapsed");
    }
    return step > 0 ? (double)io / (double)step : 1.0;
}

// Forward part of the gradient sweep: copies (and rescales) u0, runs the
// schedule up to its first adjoint step, computes u_N and E(T).  The sweep
// state stays in the context for gradient_backward.
void gradient_forward(pnop_ctx* c, const double2* u0, double E0, double horizon, double* ET, double* Einit_out) {
    Range nvtx_range("pnop:gradient_forward");
    const double dt = c->h.ph.dt;
    const double nd = horizon / dt;
    const long long N = (long long)std::llround(nd);
    if (!(horizon > 0) || N < 1 || std::fabs(nd - (double)N) > 1e-9 * std::max(1.0, nd))
        throw Status(PNOP_ERR_INVALID_ARG, "horizon must be a positive whole number of time steps");
    c->pending = false;
    if (!c->batched) {
        ensure_shadow(c);
        // work a failed earlier sweep may have left on the shadow comes first
        ck(cudaEventRecord(c->ev_shadow, c->shadow->stream), "event");
        ck(cudaStreamWaitEvent(c->stream, c->ev_shadow, 0), "wait");
    }
    const int s = snapshot_slots(c, N);
    while ((int)c->snaps.size() < s) c->snaps.push_back(c->field());
    if (!c->uN) c->uN = c->field();
    const size_t fb = c->field_bytes();
    ck(cudaMemcpyAsync(c->snaps[0], u0, fb, cudaMemcpyDeviceToDevice, c->stream), "copy u0");
    double Einit = 0.5 * inner_sync(c, c->snaps[0], c->snaps[0]);
    if (E0 > 0) {
        if (!(Einit > 0) || !std::isfinite(Einit)) throw Status(PNOP_ERR_NONFINITE, "initial field has no finite energy");
        axpby(c, std::sqrt(E0 / Einit), c->snaps[0], 0.0, nullptr, c->snaps[0]);
        Einit = 0.5 * inner_sync(c, c->snaps[0], c->snaps[0]);
    }
    c->st_adv = c->st_adj = c->st_store = 0;
    c->st_slots = s;
    c->plan.clear();
    const int nf = (c->host_max > 0 && N > 1) ? choose_host_checkpoints(N, s, c->host_max, c->host_ratio) : 0;
    c->st_nf = nf;
    c->st_hstore = c->st_hload = 0;
    if (nf > 0) {
        ensure_host_tier(c, nf);
        plan_two_level(c->plan, N, s, nf);
    } else {
        plan_reverse(c->plan, 0, N, 0, s);
    }
    const double2* st = nullptr;
    c->plan_pos = run_plan(c, 0, true, &st);
    if (c->plan_pos >= c->plan.size() || c->plan[c->plan_pos].start != N - 1)
        throw Status(PNOP_ERR_INVALID_ARG, "checkpoint schedule out of order");
    // terminal state u_N (the compatibility condition Eq. 2.8 uses it)
    fwd_step(c, st, c->uN, c->h.ph.tau0 + (N - 1) * dt);
    ++c->st_adv;
    const double ET2 = inner_sync(c, c->uN, c->uN);
    if (!std::isfinite(ET2)) throw Status(PNOP_ERR_NONFINITE, "final energy is not finite");
    *ET = 0.5 * ET2;
    if (Einit_out) *Einit_out = Einit;
    for (size_t i = c->plan_pos; i < c->plan.size(); ++i)  // start the first host load early
        if (c->plan[i].kind == kLoad) {
            host_prefetch(c, c->plan[i].host);
            break;
        }
    c->pending = true;
}

// Backward part: terminal cotangent gE * W_hat u_N, the remaining schedule,
// then grad = cotangent / W_hat (Riesz) or the Euclidean cotangent itself.
void gradient_backward(pnop_ctx* c, double gE, bool euclidean, double2* grad) {
    Range nvtx_range("pnop:gradient_backward");
    if (!c->pending) throw Status(PNOP_ERR_INVALID_ARG, "no pending gradient forward on this context");
    c->pending = false;
    weight(c, c->uN, c->lamA, 0);
    if (gE != 1.0) axpby(c, gE, c->lamA, 0.0, nullptr, c->lamA);
    const double2* st = nullptr;
    if (c->shadow && c->st_nf == 0) run_plan_overlap(c, c->plan_pos);
    else run_plan(c, c->plan_pos, false, &st);
    if (euclidean) ck(cudaMemcpyAsync(grad, c->lamA, c->field_bytes(), cudaMemcpyDeviceToDevice, c->stream), "copy");
    else weight(c, c->lamA, grad, 1);
    wait_stream(c, "gradient sync");
}

// Backward part with the continuous adjoint: w(T) = u_N (compatibility
// condition Eq. 2.8, w = -u_dagger), integrated back over the same schedule;
// w(tau0) is the gradient in the energy inner product.
void gradient_backward_continuous(pnop_ctx* c, double2* grad) {
    if (!c->pending) throw Status(PNOP_ERR_INVALID_ARG, "no pending gradient forward on this context");
    c->pending = false;
    if (!c->cprev) c->cprev = c->field();
    const size_t fb = c->field_bytes();
    ck(cudaMemcpyAsync(c->lamA, c->uN, fb, cudaMemcpyDeviceToDevice, c->stream), "terminal");
    ck(cudaMemcpyAsync(c->cprev, c->uN, fb, cudaMemcpyDeviceToDevice, c->stream), "terminal state");
    const double2* st = nullptr;
    c->continuous = true;
    try {
        run_plan(c, c->plan_pos, false, &st);
    } catch (...) {
        c->continuous = false;
        throw;
    }
    c->continuous = false;
    ck(cudaMemcpyAsync(grad, c->lamA, fb, cudaMemcpyDeviceToDevice, c->stream), "copy");
    wait_stream(c, "gradient sync");
}

int gradient_impl(pnop_ctx* c, const double2* u0, double E0, double horizon, double2* grad, double* gain) {
    double ET = 0, Einit = 0;
    gradient_forward(c, u0, E0, horizon, &ET, &Einit);
    gradient_backward(c, 1.0, false, grad);
    if (gain) *gain = ET / Einit;
    return PNOP_OK;
}

// Adjoint looping (Section 2.3).  With u_dagger = -g (g the Riesz gradient of
// E(T)), the update (1 + lambda alpha) u - alpha u_dagger = (1 + lambda alpha) u
// + alpha g keeps E = E0 for lambda = lambda_+ of Eq. 2.14 (C0 = <u, u_dagger>,
// E0_dagger = <u_dagger, u_dagger>/2), real for 0 < alpha <= alpha_max
// (Eq. 2.15).  A trial point costs the checkpointed forward sweep; when it
// raises G the reverse sweep of that same sweep gives the next gradient.
void optimise_impl(pnop_ctx* c, double2* u, double E0, double horizon, int max_iter, double tol, bool continuous,
                   double* hist, pnop_opt_stats* st) {
    constexpr int kMaxHalvings = 60;
    if (!c->opt_g) c->opt_g = c->field();
    if (!c->opt_u) c->opt_u = c->field();
    double2 *g = c->opt_g, *trial = c->opt_u;
    project(c, u);
    const double E = 0.5 * inner_sync(c, u, u);
    if (!(E > 0) || !std::isfinite(E)) throw Status(PNOP_ERR_NONFINITE, "initial field has no finite energy");
    axpby(c, std::sqrt(E0 / E), u, 0.0, nullptr, u);
    double ET = 0, Eu = 0;
    auto backward = [&] {
        if (continuous) gradient_backward_continuous(c, g);
        else gradient_backward(c, 1.0, false, g);
        project(c, g);
    };
    gradient_forward(c, u, -1.0, horizon, &ET, &Eu);
    backward();
    double G = ET / Eu;
    *st = pnop_opt_stats{0, 1, 1, 0, G, std::nan("")};
    if (hist) hist[0] = G;
    for (int it = 0; it < max_iter && !st->converged; ++it) {
        const double E0d = 0.5 * inner_sync(c, g, g);  // |u_dagger| = |g|
        const double C0 = -inner_sync(c, u, g);
        const double d = E0d / E0 - C0 * C0 / (4.0 * E0 * E0);
        if (!std::isfinite(d)) throw Status(PNOP_ERR_NONFINITE, "gradient is not finite");
        if (d <= 1e-12 * (E0d / E0)) {  // u_dagger parallel to u: the optimality condition
            st->converged = 1;
            break;
        }
        double alpha = c->opt_alpha_frac / std::sqrt(d);
        bool accepted = false;
        double Gn = G, R = 0;
        for (int h = 0; h < kMaxHalvings; ++h) {
            const double b = (alpha * C0 - 2.0 * E0) / (2.0 * alpha * E0);
            const double lam = b + std::sqrt(std::max(0.0, b * b - (alpha * E0d - C0) / (alpha * E0)));
            axpby(c, 1.0 + lam * alpha, u, alpha, g, trial);
            bool finite = true;
            try {
                gradient_forward(c, trial, -1.0, horizon, &ET, &Eu);
            } catch (const Status& e) {
                if (e.code != PNOP_ERR_NONFINITE) throw;
                finite = false;  // the trial blew up: treat as no growth
            }
            ++st->forward_evals;
            Gn = finite ? ET / Eu : std::nan("");
            R = std::isfinite(Gn) ? std::fabs(Gn - G) / std::fabs(Gn) : INFINITY;
            if (std::isfinite(Gn) && Gn > G) {
                accepted = true;
                break;
            }
            if (R < tol) break;
            alpha *= 0.5;
        }
        if (!accepted) {
            st->converged = 1;
            break;
        }
        backward();
        ++st->gradients;
        ck(cudaMemcpyAsync(u, trial, c->field_bytes(), cudaMemcpyDeviceToDevice, c->stream), "accept");
        G = Gn;
        st->iterations = it + 1;
        st->gain = G;
        st->rel_change = R;
        if (hist) hist[it + 1] = G;
        if (R < tol) st->converged = 1;
    }
    c->pending = false;  // the last trial's sweep is not the caller's
    wait_stream(c, "optimise sync");
}

// ------------------------------------------------------------------ batched gradients
// A batched context runs the checkpointed gradient of up to nslot requests of
// one grid, each with its own Re, Wo, A, dt, tau0, E0 and horizon.  Each
// request turns its binomial schedule (Section 2.5) into a queue of per-slot
// operations; a tick takes every request to its next step and launches one
// batched forward, terminal or adjoint step for all requests whose next step
// is of the kind most of them wait for.  The steps are the same
// predictor-corrector step and its exact transpose as the single-request
// path, in place on the slot's state and cotangent, so every request gets
// bitwise the gradient it gets alone.

// Active batch entries of the next launches: geo.nb and geo.slot.
void batch_select(pnop_ctx* c, const std::vector<int>& slots) {
    Geo& g = c->geo;
    g.nb = (int)slots.size();
    for (int b = 0; b < g.nb; ++b) g.slot[b] = slots[b];
}
void batch_reset(pnop_ctx* c) {
    c->geo.nb = 1;
    c->geo.slot[0] = 0;
}

double2* slot_ptr(pnop_ctx* c, double2* base, int slot) { return base + (size_t)slot * 3 * c->S(); }

// Queue of operations of one request from its binomial plan: the first
// adjoint step (N - 1) is preceded by the terminal step u_{N-1} -> u_N.
void batch_ops(BatchReq& r, const std::vector<Action>& P) {
    r.ops.clear();
    bool first_adj = true;
    for (const Action& a : P) {
        if (a.kind == kAdv) {
            r.ops.push_back({kOpRestore, 0, a.slot});
            for (long long i = 0; i < a.n; ++i) r.ops.push_back({kOpFwd, a.start + i, -1});
            if (a.dst >= 0) r.ops.push_back({kOpStore, 0, a.dst});
        } else if (a.kind == kAdj) {
            if (a.slot >= 0) r.ops.push_back({kOpRestore, 0, a.slot});
            if (first_adj) {
                if (a.start != r.N - 1) throw Status(PNOP_ERR_INVALID_ARG, "checkpoint schedule out of order");
                r.ops.push_back({kOpTerm, r.N - 1, -1});
                first_adj = false;
            }
            r.ops.push_back({kOpAdj, a.start, -1});
        } else {
            throw Status(PNOP_ERR_UNSUPPORTED, "host checkpoints are not used by batched contexts");
        }
    }
    r.ops.push_back({kOpFinish, 0, -1});
    r.pos = 0;
}

// Host operators of one request's physics on the batch's grid.  Reads only the
// batch's grid tables and pressure factors (fixed after creation), so any
// number of these can run at once, beside the batch's other calls.
pnop::HostOps batch_prepare(const pnop_ctx* c, const pnop_params* p) {
    if (!p || !(p->Re > 0) || !(p->dt > 0) || !(p->A >= 0) || !(p->Wo > 0 || p->A == 0))
        throw Status(PNOP_ERR_INVALID_ARG, "bad request parameters");
    pnop::HostOps hs;
    hs.d = c->h.d;
    hs.r = c->h.r;
    hs.invr = c->h.invr;
    hs.W = c->h.W;
    hs.D1 = c->h.D1;
    hs.D2 = c->h.D2;
    hs.facP = c->h.facP;
    hs.facPT = c->h.facPT;
    hs.ph = {p->Re, p->Wo, p->A, p->dt, p->tau0};
    std::string err;
    if (!pnop::build_operators(hs, err, true)) throw Status(PNOP_ERR_UNSUPPORTED, err);
    return hs;
}

int batch_submit(pnop_ctx* c, const pnop::HostOps& hs, const double2* u0, double E0, double horizon) {
    const pnop::Physics* p = &hs.ph;
    if (!u0) throw Status(PNOP_ERR_INVALID_ARG, "u0 is NULL");
    if (hs.d.nr != c->h.d.nr || hs.d.M != c->h.d.M || hs.d.K != c->h.d.K || hs.d.Lz != c->h.d.Lz ||
        hs.d.stretch != c->h.d.stretch)
        throw Status(PNOP_ERR_INVALID_ARG, "operators prepared for another grid");
    const double nd = horizon / p->dt;
    const long long N = (long long)std::llround(nd);
    if (!(horizon > 0) || N < 1 || std::fabs(nd - (double)N) > 1e-9 * std::max(1.0, nd))
        throw Status(PNOP_ERR_INVALID_ARG, "horizon must be a positive whole number of time steps");
    int slot = -1;
    for (int i = 0; i < c->nslot; ++i)
        if (!c->breq[i].active && c->breq[i].fetched) {
            slot = i;
            break;
        }
    if (slot < 0) throw Status(PNOP_ERR_OOM, "no free slot in the batch");
    // operators of this request's physics into the slot's tables (the slot
    // is idle: no queued launch reads them)
    upload_slot_operators(c, slot, hs);
    const int s = (int)std::max<long long>(1, std::min<long long>(c->prm.snap_budget, N));
    while ((int)c->snaps.size() < s) c->snaps.push_back(c->field());
    BatchReq& r = c->breq[slot];
    r.Re = p->Re;
    r.Wo = p->Wo;
    r.A = p->A;
    r.dt = p->dt;
    r.tau0 = p->tau0;
    r.omega = hs.omega;
    r.E0 = E0;
    r.N = N;
    std::vector<Action> P;
    plan_reverse(P, 0, N, 0, s);
    batch_ops(r, P);
    if (!r.ev_done) ck(cudaEventCreateWithFlags(&r.ev_done, cudaEventDisableTiming), "event");
    // u0 into checkpoint 0, scaled to E0 on the device (as the single path does on the host)
    double2* s0 = slot_ptr(c, c->snaps[0], slot);
    ck(cudaMemcpyAsync(s0, u0, c->field_bytes(), cudaMemcpyDeviceToDevice, c->stream), "copy u0");
    batch_select(c, {slot});
    inner_dev(c, c->snaps[0], c->snaps[0], c->d_e0);
    if (E0 > 0) {
        run(c, PNOP_K_ELEMENTWISE, 1, 3.0 * c->S(),
            [&] { pnop::launch_scale_energy(c->geo, c->snaps[0], E0, 0.5, c->d_e0, c->stream); });
        inner_dev(c, c->snaps[0], c->snaps[0], c->d_e0);
    }
    batch_reset(c);
    r.id = c->next_id++;
    r.active = true;
    r.done = false;
    r.fetched = false;
    return r.id;
}

// One tick: copies and finished requests first, then one batched step.
// Returns false when no request has work left.
bool batch_tick(pnop_ctx* c) {
    Range nvtx_range("pnop:batch_tick");
    std::vector<int> lists[3], fin;  // kOpFwd, kOpTerm, kOpAdj
    const size_t fb = c->field_bytes();
    for (int i = 0; i < c->nslot; ++i) {
        BatchReq& r = c->breq[i];
        if (!r.active || r.done) continue;
        while (r.pos < r.ops.size() && (r.ops[r.pos].kind == kOpRestore || r.ops[r.pos].kind == kOpStore)) {
            const Op& o = r.ops[r.pos++];
            double2* st = slot_ptr(c, c->bcur, i);
            double2* ck_ = slot_ptr(c, c->snaps[o.snap], i);
            if (o.kind == kOpRestore) ck(cudaMemcpyAsync(st, ck_, fb, cudaMemcpyDeviceToDevice, c->stream), "restore");
            else ck(cudaMemcpyAsync(ck_, st, fb, cudaMemcpyDeviceToDevice, c->stream), "store");
        }
        const int k = r.ops[r.pos].kind;
        if (k == kOpFinish) fin.push_back(i);
        else lists[k - kOpFwd].push_back(i);
    }
    if (!fin.empty()) {  // gradient = W_hat^-1 cotangent (Riesz), into the slot's result field
        batch_select(c, fin);
        weight(c, c->blam, c->uN, 1);
        batch_reset(c);
        for (int i : fin) {
            BatchReq& r = c->breq[i];
            ck(cudaEventRecord(r.ev_done, c->stream), "record");
            r.done = true;
            ++r.pos;
        }
    }
    // the kind with most waiting requests (ties: adjoint, forward, terminal)
    int kind = -1;
    size_t best = 0;
    for (int k : {2, 0, 1})
        if (lists[k].size() > best) {
            best = lists[k].size();
            kind = k;
        }
    if (kind < 0) return !fin.empty();
    const std::vector<int>& sel = lists[kind];
    batch_select(c, sel);
    for (int b = 0; b < (int)sel.size(); ++b) {
        const BatchReq& r = c->breq[sel[b]];
        c->bt[b] = r.tau0 + r.ops[r.pos].n * r.dt;
    }
    if (kind == 0) {
        fwd_step(c, c->bcur, c->bcur, 0.0);
        c->st_adv += (long long)sel.size();
    } else if (kind == 1) {  // terminal step, its energy, and the terminal cotangent W_hat u_N
        fwd_step(c, c->bcur, c->uN, 0.0);
        inner_dev(c, c->uN, c->uN, c->d_eT);
        weight(c, c->uN, c->blam, 0);
        c->st_adv += (long long)sel.size();
    } else {
        adj_step(c, c->bcur, 0.0, c->blam, c->blam);
        c->st_adj += (long long)sel.size();
    }
    batch_reset(c);
    for (int i : sel) ++c->breq[i].pos;
    ++c->b_ticks;
    c->b_launch_entries += (long long)sel.size();
    return true;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* pnop_error_string(int status) {
    switch (status) {
        case PNOP_OK: return "ok";
        case PNOP_ERR_INVALID_ARG: return "invalid argument";
        case PNOP_ERR_OOM: return "out of device memory or HBM budget";
        case PNOP_ERR_CUDA: return "CUDA error";
        case PNOP_ERR_NONFINITE: return "non-finite result";
        case PNOP_ERR_TIMEOUT: return "timeout";
        case PNOP_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

const char* pnop_last_error(const pnop_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int pnop_context_bytes(const pnop_grid* grid, const pnop_params* params, int snaps, size_t* bytes) {
    if (!grid || !params || !bytes || snaps < 1 || grid->nr < 1 || grid->ntheta < 4 || grid->nz < 4)
        return PNOP_ERR_INVALID_ARG;
    const size_t nr = grid->nr, M = grid->ntheta / 2 - 1, K = grid->nz / 2 - 1;
    const size_t nm = 2 * M + 1, nk = K + 1, nkp = (nk + pnop::kTileK - 1) / pnop::kTileK * pnop::kTileK, nt = 3 * (M + 1);
    const size_t S = nr * nm * nk, field = 3 * S * 16;
    const size_t cz = (params->precision & PNOP_MIXED) ? 8 : 16;
    size_t b = (21 + (size_t)snaps) * field + 2 * S * 16;              // work fields, u_N, optimiser, host staging, checkpoints, q, q2
    b += 24 * nr * nt * nk * cz;                                         // transform scratch Y, Y2, Z
    b += 10 * field + S * 16 + 15 * nr * nt * nk * cz;                   // recomputation workspace (shadow) and its scratch states
    b += 2 * ((M + 2) + (M + 1)) * nr * 13 * nkp * 8;                    // LU factors and transposed rows
    b += (M + 2) * nr * 13 * 8 + 2 * nr * 13 * 8 + nm * nk * 3 * nr * 8; // bands, D1, influence
    *bytes = b + (1 << 20) + (40 + (size_t)snaps) * (2 << 20);        // tables, reductions, allocation rounding
    return PNOP_OK;
}

int pnop_device_bytes(const pnop_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return PNOP_ERR_INVALID_ARG;
    *bytes = ctx->bytes;
    return PNOP_OK;
}

int pnop_batch_bytes(const pnop_grid* grid, const pnop_params* params, int capacity, size_t* bytes) {
    if (!grid || !params || !bytes || params->snap_budget < 1 || capacity < 1 || capacity > pnop::kMaxBatch ||
        grid->nr < 1 || grid->ntheta < 4 || grid->nz < 4)
        return PNOP_ERR_INVALID_ARG;
    const size_t nr = grid->nr, M = grid->ntheta / 2 - 1, K = grid->nz / 2 - 1, C = capacity;
    const size_t nm = 2 * M + 1, nk = K + 1, nkp = (nk + pnop::kTileK - 1) / pnop::kTileK * pnop::kTileK, nt = 3 * (M + 1);
    const size_t S = nr * nm * nk, field = 3 * S * 16, snaps = (size_t)params->snap_budget;
    const size_t cz = (params->precision & PNOP_MIXED) ? 8 : 16;
    size_t b = C * (18 + snaps) * field;                                 // work fields, state, cotangent, result, q, q2, checkpoints
    b += C * 27 * nr * nt * nk * cz;                                     // transform scratch Y, Y2, Z (9 planes each)
    b += C * 2 * (M + 2) * nr * 13 * nkp * 8 + 2 * (M + 1) * nr * 13 * nkp * 8;  // Helmholtz factors per slot, pressure shared
    b += C * ((M + 2) * nr * 13 * 8 + nm * nk * 3 * nr * 8 + nk * 8 + 5 * nr * 8) + 2 * nr * 13 * 8;  // bands, influence
    *bytes = b + (1 << 20) + C * (40 + snaps) * (2 << 20);              // tables, reductions, allocation rounding
    return PNOP_OK;
}

int pnop_two_level_counts(long long nsteps, int snaps, long long max_host_slots, double io_ratio,
                          int* host_checkpoints, long long* advances) {
    if (nsteps < 1 || snaps < 1 || max_host_slots < 0 || !(io_ratio >= 0) || !std::isfinite(io_ratio))
        return PNOP_ERR_INVALID_ARG;
    const int s = (int)std::min<long long>(snaps, nsteps);
    const int nf = nsteps > 1 ? choose_host_checkpoints(nsteps, s, max_host_slots, io_ratio) : 0;
    if (host_checkpoints) *host_checkpoints = nf;
    if (advances) *advances = (long long)std::llround(two_level_steps(nsteps, s, nf));
    return PNOP_OK;
}

int pnop_revolve_counts(int nsteps, int snaps, long long* advances, long long* stores) {
    if (nsteps < 1 || snaps < 1) return PNOP_ERR_INVALID_ARG;
    long long adv = 0, st = 0;
    count_reverse(nsteps, snaps, adv, st);
    if (advances) *advances = adv;
    if (stores) *stores = st;
    return PNOP_OK;
}

void pnop_destroy(pnop_ctx* ctx) {
    if (!ctx) return;
    if (ctx->shadow) {
        cudaStreamSynchronize(ctx->shadow->stream);
        pnop_destroy(ctx->shadow);
    }
    for (cudaEvent_t e : {ctx->ev_ring_w[0], ctx->ev_ring_w[1], ctx->ev_ring_r[0], ctx->ev_ring_r[1], ctx->ev_main,
                          ctx->ev_shadow})
        if (e) cudaEventDestroy(e);
    for (auto e : ctx->ev_slot_w)
        if (e) cudaEventDestroy(e);
    for (auto e : ctx->ev_slot_r)
        if (e) cudaEventDestroy(e);
    for (auto e : ctx->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_t, ctx->ev_base})
        if (e) cudaEventDestroy(e);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->copy) {
        cudaStreamSynchronize(ctx->copy);
        cudaStreamDestroy(ctx->copy);
    }
    for (cudaEvent_t e : {ctx->ev_copy, ctx->ev_staged})
        if (e) cudaEventDestroy(e);
    for (void* p : ctx->host) cudaFreeHost(p);
    for (auto& r : ctx->breq)
        if (r.ev_done) cudaEventDestroy(r.ev_done);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->owns_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"

namespace {
// A context with nslot storage slots (1: the single-request context of
// pnop_create; batched: pnop_batch_create, one request per slot).
int create_impl(const pnop_grid* grid, const pnop_params* params, void* cuda_stream, int nslot, bool batched,
                pnop_ctx** out) {
    if (!out) return PNOP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !params || nslot < 1 || nslot > pnop::kMaxBatch) return PNOP_ERR_INVALID_ARG;
    if (grid->nr < 9 || grid->ntheta < 4 || grid->nz < 4 || (grid->ntheta & 1) || (grid->nz & 1) ||
        !(grid->Lz > 0) || !(grid->stretch >= 0 && grid->stretch < 1))
        return PNOP_ERR_INVALID_ARG;
    if (!(params->Re > 0) || !(params->dt > 0) ||
        params->precision < PNOP_FP64 || params->precision > PNOP_MIXED_DF || !(params->A >= 0) ||
        !(params->Wo > 0 || params->A == 0))
        return PNOP_ERR_INVALID_ARG;
    const int M = grid->ntheta / 2 - 1, K = grid->nz / 2 - 1;
    if (!smooth_size(3 * (M + 1)) || !smooth_size(3 * (K + 1))) return PNOP_ERR_UNSUPPORTED;
    pnop_ctx* c = new pnop_ctx();
    c->prm = *params;
    c->stream = (cudaStream_t)cuda_stream;
    c->nslot = nslot;
    c->batched = batched;
    pnop::Dims& d = c->h.d;
    d.nr = grid->nr;
    d.M = M;
    d.K = K;
    d.nm = 2 * M + 1;
    d.nk = K + 1;
    d.nth = 3 * (M + 1);
    d.nzp = 3 * (K + 1);
    d.Lz = grid->Lz;
    d.stretch = grid->stretch;
    c->h.ph = {params->Re, params->Wo, params->A, params->dt, params->tau0};
    int rc = guarded(c, [&]() -> int {
        std::string err;
        if (!pnop::build_grid(c->h, err)) throw Status(PNOP_ERR_UNSUPPORTED, err);
        if (!pnop::build_operators(c->h, err)) throw Status(PNOP_ERR_UNSUPPORTED, err);
        Geo& g = c->geo;
        g.nr = d.nr;
        g.M = M;
        g.K = K;
        g.nm = d.nm;
        g.nk = d.nk;
        g.nt = d.nth;
        g.nzp = d.nzp;
        g.kz0 = 2.0 * M_PI / d.Lz;
        g.ewt = 2.0 * M_PI * d.Lz;
        g.nb = 1;
        g.slot[0] = 0;
        g.fs = 3 * c->S();
        c->d_r = c->upload(c->h.r);
        c->d_invr = c->upload(c->h.invr);
        c->d_W = c->upload(c->h.W);
        c->d_D1 = c->upload(c->h.D1);
        g.r = c->d_r;
        g.invr = c->d_invr;
        g.W = c->d_W;
        g.D1 = c->d_D1;
        {
            std::vector<double> kz(d.nk), mr((size_t)d.nm * d.nr);
            for (int k = 0; k < d.nk; ++k) kz[k] = k * g.kz0;
            for (int im = 0; im < d.nm; ++im)
                for (int j = 0; j < d.nr; ++j) mr[(size_t)im * d.nr + j] = (im - M) * c->h.invr[j];
            g.kzt = c->upload(kz);
            g.mrt = c->upload(mr);
            g.df = (params->precision & PNOP_DF) ? 1 : 0;
            if (g.df) {
                g.D1f = c->upload(split_pairs(c->h.D1));
                g.invrf = c->upload(split_pairs(c->h.invr));
                g.kztf = c->upload(split_pairs(kz));
                g.mrtf = c->upload(split_pairs(mr));
            }
        }
        upload_operators(c);
        auto thd = twiddle_table<double2>(d.nth), zd = twiddle_table<double2>(d.nzp);
        auto thf = twiddle_table<float2>(d.nth), zf = twiddle_table<float2>(d.nzp);
        c->tw.th_d = c->upload(thd);
        c->tw.z_d = c->upload(zd);
        c->tw.th_f = c->upload(thf);
        c->tw.z_f = c->upload(zf);
        for (double2** b : {&c->omega, &c->N0, &c->N1, &c->us, &c->ua, &c->Fb, &c->Nb, &c->ubs, &c->wb, &c->R,
                            &c->Rl, &c->Nbase})
            *b = c->field();
        c->ac = (double2*)c->dalloc((size_t)nslot * d.nm * d.nk * sizeof(double2));
        c->pw = (double*)c->dalloc((size_t)nslot * 3 * d.nm * d.nk * sizeof(double2));
        if (batched) {  // per-slot state, cotangent and energies replace the sweep buffers
            c->bcur = c->field();
            c->blam = c->field();
            c->uN = c->field();  // terminal state, then the finished gradient
            c->d_e0 = (double*)c->dalloc(nslot * sizeof(double));
            c->d_eT = (double*)c->dalloc(nslot * sizeof(double));
            c->breq.resize(nslot);
        } else {
            for (double2** b : {&c->tmpA, &c->tmpB, &c->lamA, &c->lamB}) *b = c->field();
        }
        // one-component scratch: a full field per slot when batched (the slot stride is 3 S)
        c->q = batched ? c->field() : (double2*)c->dalloc(c->S() * sizeof(double2));
        c->q2 = batched ? c->field() : (double2*)c->dalloc(c->S() * sizeof(double2));
        ck(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
        for (cudaEvent_t* e : {&c->ev_fork, &c->ev_t, &c->ev_base})
            ck(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event");
        const size_t cz = mixed(c) ? sizeof(float2) : sizeof(double2);
        const size_t plane = (size_t)d.nr * d.nth * d.nk * cz;
        g.ps = 9 * (size_t)d.nr * d.nth * d.nk;  // physical planes per slot (elements)
        c->Y = c->dalloc(nslot * 9 * plane);
        c->Y2 = c->dalloc(nslot * 9 * plane);
        c->Z = c->dalloc((batched ? nslot * 9 : 6) * plane);
        c->partial = (double*)c->dalloc(nslot * pnop::inner_partials(g) * sizeof(double));
        c->dscal = (double*)c->dalloc(4 * sizeof(double));
        if (batched) c->h.ph.dt = 1.0;  // batched steps take times as step offsets (set_phase)
        ck(cudaDeviceSynchronize(), "create");
        return PNOP_OK;
    });
    if (rc != PNOP_OK) {
        pnop_destroy(c);
        return rc;
    }
    *out = c;
    return PNOP_OK;
}
}  // namespace

extern "C" {

int pnop_create(const pnop_grid* grid, const pnop_params* params, void* cuda_stream, pnop_ctx** out) {
    return create_impl(grid, params, cuda_stream, 1, false, out);
}

int pnop_set_base_flow(pnop_ctx* ctx, double Re, double Wo, double A, double tau0) {
    return guarded(ctx, [&]() -> int {
        ctx->pending = false;  // shares the sweep buffers
        if (!(Re > 0) || !(A >= 0) || !(Wo > 0 || A == 0)) throw Status(PNOP_ERR_INVALID_ARG, "bad base-flow parameters");
        ctx->h.ph.Re = Re;
        ctx->h.ph.Wo = Wo;
        ctx->h.ph.A = A;
        ctx->h.ph.tau0 = tau0;
        ctx->prm.Re = Re;
        ctx->prm.Wo = Wo;
        ctx->prm.A = A;
        ctx->prm.tau0 = tau0;
        std::string err;
        ck(cudaStreamSynchronize(ctx->stream), "sync");
        if (!pnop::build_operators(ctx->h, err)) throw Status(PNOP_ERR_UNSUPPORTED, err);
        upload_operators(ctx);
        return PNOP_OK;
    });
}

int pnop_dims(const pnop_ctx* ctx, int* nr, int* M, int* K) {
    if (!ctx) return PNOP_ERR_INVALID_ARG;
    if (nr) *nr = ctx->h.d.nr;
    if (M) *M = ctx->h.d.M;
    if (K) *K = ctx->h.d.K;
    return PNOP_OK;
}

int pnop_grid_points(const pnop_ctx* ctx, double* r_out) {
    if (!ctx || !r_out) return PNOP_ERR_INVALID_ARG;
    std::memcpy(r_out, ctx->h.r.data(), ctx->h.r.size() * sizeof(double));
    return PNOP_OK;
}

int pnop_step_forward(pnop_ctx* ctx, void* u, double t, int nsteps) {
    return guarded(ctx, [&]() -> int {
        ctx->pending = false;  // shares the sweep buffers
        if (!u || nsteps < 0) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        double2* uu = (double2*)u;
        for (int i = 0; i < nsteps; ++i) {
            fwd_step(ctx, uu, ctx->tmpA, t + i * ctx->h.ph.dt);
            ck(cudaMemcpyAsync(uu, ctx->tmpA, ctx->field_bytes(), cudaMemcpyDeviceToDevice, ctx->stream), "copy");
        }
        ck(cudaGetLastError(), "step_forward");
        return PNOP_OK;
    });
}

int pnop_step_adjoint(pnop_ctx* ctx, const void* u_n, void* lam, double t_n) {
    return guarded(ctx, [&]() -> int {
        ctx->pending = false;  // shares the sweep buffers
        if (!u_n || !lam) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        double2* l = (double2*)lam;
        weight(ctx, l, ctx->tmpA, 0);
        adj_step(ctx, (const double2*)u_n, t_n, ctx->tmpA, ctx->tmpB);
        weight(ctx, ctx->tmpB, l, 1);
        ck(cudaGetLastError(), "step_adjoint");
        return PNOP_OK;
    });
}

int pnop_gradient(pnop_ctx* ctx, const void* u0, double E0, double horizon, void* grad_out, double* gain_out) {
    return guarded(ctx, [&]() -> int {
        if (!u0 || !grad_out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        return gradient_impl(ctx, (const double2*)u0, E0, horizon, (double2*)grad_out, gain_out);
    });
}

int pnop_gradient_continuous(pnop_ctx* ctx, const void* u0, double E0, double horizon, void* grad_out,
                             double* gain_out) {
    return guarded(ctx, [&]() -> int {
        if (!u0 || !grad_out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        double ET = 0, Einit = 0;
        gradient_forward(ctx, (const double2*)u0, E0, horizon, &ET, &Einit);
        gradient_backward_continuous(ctx, (double2*)grad_out);
        if (gain_out) *gain_out = ET / Einit;
        return PNOP_OK;
    });
}

int pnop_gradient_forward(pnop_ctx* ctx, const void* u0, double E0, double horizon, double* ET_out, double* E0_out) {
    return guarded(ctx, [&]() -> int {
        if (!u0 || !ET_out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        gradient_forward(ctx, (const double2*)u0, E0, horizon, ET_out, E0_out);
        return PNOP_OK;
    });
}

int pnop_gradient_backward(pnop_ctx* ctx, double gE, int euclidean, void* grad_out) {
    return guarded(ctx, [&]() -> int {
        if (!grad_out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        gradient_backward(ctx, gE, euclidean != 0, (double2*)grad_out);
        return PNOP_OK;
    });
}

int pnop_gradient_host(pnop_ctx* ctx, const double* u0_host, double E0, double horizon, double* grad_host,
                       double* gain_out) {
    return guarded(ctx, [&]() -> int {
        if (!u0_host || !grad_host) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        const size_t fb = ctx->field_bytes();
        ck(cudaMemcpyAsync(ctx->tmpA, u0_host, fb, cudaMemcpyHostToDevice, ctx->stream), "h2d");
        // tmpA is reused by the sweep: stage the input in the gradient output slot of lamB
        ck(cudaMemcpyAsync(ctx->lamB, ctx->tmpA, fb, cudaMemcpyDeviceToDevice, ctx->stream), "stage");
        int rc = gradient_impl(ctx, ctx->lamB, E0, horizon, ctx->tmpB, gain_out);
        if (rc != PNOP_OK) return rc;
        ck(cudaMemcpyAsync(grad_host, ctx->tmpB, fb, cudaMemcpyDeviceToHost, ctx->stream), "d2h");
        ck(cudaStreamSynchronize(ctx->stream), "sync");
        return PNOP_OK;
    });
}

int pnop_optimise_ex(pnop_ctx* ctx, void* u0, double E0, double horizon, int max_iter, double tol, int adjoint,
                     double* gain_history, pnop_opt_stats* stats) {
    return guarded(ctx, [&]() -> int {
        if (!u0 || !(E0 > 0) || max_iter < 0 || !(tol >= 0) ||
            (adjoint != PNOP_ADJOINT_DISCRETE && adjoint != PNOP_ADJOINT_CONTINUOUS))
            throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        pnop_opt_stats st{};
        optimise_impl(ctx, (double2*)u0, E0, horizon, max_iter, tol, adjoint == PNOP_ADJOINT_CONTINUOUS,
                      gain_history, &st);
        if (stats) *stats = st;
        return PNOP_OK;
    });
}

int pnop_optimise(pnop_ctx* ctx, void* u0, double E0, double horizon, int max_iter, double tol,
                  double* gain_history, pnop_opt_stats* stats) {
    return pnop_optimise_ex(ctx, u0, E0, horizon, max_iter, tol, PNOP_ADJOINT_DISCRETE, gain_history, stats);
}

int pnop_mode_energy(pnop_ctx* ctx, const void* u, double* spectrum) {
    return guarded(ctx, [&]() -> int {
        if (!u || !spectrum) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        const size_t n = 2 * (size_t)ctx->geo.nm * ctx->geo.nk;
        if (!ctx->d_spec) ctx->d_spec = (double*)ctx->dalloc(n * sizeof(double));
        run(ctx, PNOP_K_REDUCE, 1, 3.0 * ctx->S(),
            [&] { pnop::launch_mode_energy(ctx->geo, (const double2*)u, ctx->d_spec, ctx->stream); });
        ck(cudaMemcpyAsync(spectrum, ctx->d_spec, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy");
        wait_stream(ctx, "mode energy");
        return PNOP_OK;
    });
}

int pnop_resolution(pnop_ctx* ctx, const void* u, double E0, double* e_M, double* e_K) {
    return guarded(ctx, [&]() -> int {
        if (!u || !e_M || !e_K || !std::isfinite(E0)) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        if (!ctx->d_spec) ctx->d_spec = (double*)ctx->dalloc(2 * (size_t)ctx->geo.nm * ctx->geo.nk * sizeof(double));
        const double2* f = (const double2*)u;
        run(ctx, PNOP_K_REDUCE, 1, 3.0 * ctx->h.d.nr * (2.0 * ctx->geo.nk + ctx->geo.nm),
            [&] { pnop::launch_resolution(ctx->geo, f, ctx->d_spec, ctx->stream); });
        double ref = E0;
        if (!(E0 > 0)) {
            inner_dev(ctx, f, f, ctx->dscal);
            ck(cudaMemcpyAsync(&ref, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy");
        }
        double e[2] = {0, 0};
        ck(cudaMemcpyAsync(e, ctx->d_spec, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy");
        wait_stream(ctx, "resolution");
        if (!(E0 > 0)) ref *= 0.5;
        if (!(ref > 0) || !std::isfinite(ref) || !std::isfinite(e[0]) || !std::isfinite(e[1]))
            throw Status(PNOP_ERR_NONFINITE, "resolution: no finite positive reference energy");
        *e_M = e[0] / ref;
        *e_K = e[1] / ref;
        return PNOP_OK;
    });
}

int pnop_set_host_tier(pnop_ctx* ctx, long long max_host_slots, double io_ratio) {
    return guarded(ctx, [&]() -> int {
        if (max_host_slots < 0 || !std::isfinite(io_ratio) || max_host_slots > (1LL << 30))
            throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        ctx->pending = false;  // measuring uses the sweep buffers
        ctx->host_max = max_host_slots;
        ctx->host_ratio = io_ratio >= 0 ? io_ratio : (max_host_slots > 0 ? measure_io_ratio(ctx) : 0.0);
        return PNOP_OK;
    });
}

int pnop_host_tier_stats(const pnop_ctx* ctx, int* host_checkpoints, long long* host_stores, long long* host_loads,
                         double* io_ratio) {
    if (!ctx) return PNOP_ERR_INVALID_ARG;
    if (host_checkpoints) *host_checkpoints = ctx->st_nf;
    if (host_stores) *host_stores = ctx->st_hstore;
    if (host_loads) *host_loads = ctx->st_hload;
    if (io_ratio) *io_ratio = ctx->host_ratio;
    return PNOP_OK;
}

int pnop_gradient_stats(const pnop_ctx* ctx, long long* advances, long long* adjoint_steps, long long* stores) {
    if (!ctx) return PNOP_ERR_INVALID_ARG;
    if (advances) *advances = ctx->st_adv;
    if (adjoint_steps) *adjoint_steps = ctx->st_adj;
    if (stores) *stores = ctx->st_store;
    return PNOP_OK;
}

int pnop_apply(pnop_ctx* ctx, int op, const void* a, const void* b, void* out, double t) {
    return guarded(ctx, [&]() -> int {
        ctx->pending = false;  // shares the sweep buffers
        if (!a || !out || a == out || (b && b == out)) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        const double2* A = (const double2*)a;
        const double2* B = (const double2*)b;
        double2* O = (double2*)out;
        const Geo& g = ctx->geo;
        switch (op) {
            case PNOP_OP_CURL: run(ctx, PNOP_K_SPECTRAL, 1, flops::curl * ctx->S(), [&] { pnop::launch_curl(g, A, O, ctx->stream); }); break;
            case PNOP_OP_NONLINEAR: nonlinear(ctx, A, t, O, ctx->Y); break;
            case PNOP_OP_STAGE:
                if (!B) throw Status(PNOP_ERR_INVALID_ARG, "stage needs a forcing field");
                stage_u(ctx, A, B, O);
                break;
            case PNOP_OP_NONLINEAR_T:
                if (!B) throw Status(PNOP_ERR_INVALID_ARG, "transpose needs a cotangent field");
                nonlinearT(ctx, A, t, B, O, ctx->Y, false);
                break;
            case PNOP_OP_STAGE_T_U: stageT(ctx, A, O, 0, ctx->Fb); break;
            case PNOP_OP_STAGE_T_F: stageT(ctx, A, ctx->ua, 0, O); break;
            case PNOP_OP_NONLINEAR_ADJ:
                if (!B) throw Status(PNOP_ERR_INVALID_ARG, "b (the adjoint field) is required");
                nonlinear_adj(ctx, B, A, t, O);
                break;
            case PNOP_OP_PROJECT:
                ck(cudaMemcpyAsync(O, A, ctx->field_bytes(), cudaMemcpyDeviceToDevice, ctx->stream), "copy");
                project(ctx, O);
                break;
            default: throw Status(PNOP_ERR_INVALID_ARG, "unknown operator");
        }
        wait_stream(ctx, "apply");
        return PNOP_OK;
    });
}

int pnop_set_optimiser_first_step(pnop_ctx* ctx, double alpha_frac) {
    if (!ctx || !(alpha_frac > 0.0 && alpha_frac <= 1.0)) return PNOP_ERR_INVALID_ARG;
    ctx->opt_alpha_frac = alpha_frac;
    return PNOP_OK;
}

int pnop_set_timeout(pnop_ctx* ctx, double seconds) {
    if (!ctx || !(seconds >= 0)) return PNOP_ERR_INVALID_ARG;
    ctx->timeout_s = seconds;
    return PNOP_OK;
}

int pnop_sync(pnop_ctx* ctx) {
    return guarded(ctx, [&]() -> int {
        ck(cudaStreamSynchronize(ctx->stream), "sync");
        ck(cudaStreamSynchronize(ctx->side), "sync");
        return PNOP_OK;
    });
}

int pnop_profile(pnop_ctx* ctx, unsigned class_mask) {
    return guarded(ctx, [&]() -> int {
        prof_flush(ctx);
        ctx->prof_mask = class_mask;
        for (int i = 0; i < PNOP_K_NCLASS; ++i) {
            ctx->prof_ms[i] = 0;
            ctx->launches[i] = 0;
            ctx->units[i] = 0;
        }
        return PNOP_OK;
    });
}

int pnop_profile_read(pnop_ctx* ctx, double* ms, long long* launches, double* units) {
    return guarded(ctx, [&]() -> int {
        prof_flush(ctx);
        for (int i = 0; i < PNOP_K_NCLASS; ++i) {
            if (ms) ms[i] = ctx->prof_ms[i];
            if (launches) launches[i] = ctx->launches[i];
            if (units) units[i] = ctx->units[i];
        }
        return PNOP_OK;
    });
}

int pnop_energy(pnop_ctx* ctx, const void* u, double* E_out) {
    return guarded(ctx, [&]() -> int {
        if (!u || !E_out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        *E_out = 0.5 * inner_sync(ctx, (const double2*)u, (const double2*)u);
        return PNOP_OK;
    });
}

// ---------------------------------------------------------------- batched gradients
static pnop_ctx* bctx(pnop_batch* b) { return reinterpret_cast<pnop_ctx*>(b); }
static const pnop_ctx* bctx_c(const pnop_batch* b) { return reinterpret_cast<const pnop_ctx*>(b); }

int pnop_batch_create(const pnop_grid* grid, const pnop_params* params, int capacity, void* cuda_stream,
                      pnop_batch** out) {
    if (!out) return PNOP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || params->snap_budget < 1 || capacity < 1 || capacity > pnop::kMaxBatch) return PNOP_ERR_INVALID_ARG;
    pnop_ctx* c = nullptr;
    int rc = create_impl(grid, params, cuda_stream, capacity, true, &c);
    if (rc != PNOP_OK) return rc;
    rc = guarded(c, [&]() -> int {  // the checkpoints of every slot, so that admission allocates nothing
        while ((int)c->snaps.size() < params->snap_budget) c->snaps.push_back(c->field());
        return PNOP_OK;
    });
    if (rc != PNOP_OK) {
        pnop_destroy(c);
        return rc;
    }
    *out = reinterpret_cast<pnop_batch*>(c);
    return PNOP_OK;
}

struct pnop_ops {
    pnop::HostOps h;
};

int pnop_batch_prepare(const pnop_batch* batch, const pnop_params* request, pnop_ops** out) {
    if (!out) return PNOP_ERR_INVALID_ARG;
    *out = nullptr;
    const pnop_ctx* c = bctx_c(batch);
    if (!c) return PNOP_ERR_INVALID_ARG;
    try {  // records no error text: the batch may be in use by another thread
        pnop_ops* o = new pnop_ops();
        try {
            o->h = batch_prepare(c, request);
        } catch (...) {
            delete o;
            throw;
        }
        *out = o;
        return PNOP_OK;
    } catch (const Status& s) {
        return s.code;
    } catch (const std::bad_alloc&) {
        return PNOP_ERR_OOM;
    } catch (...) {
        return PNOP_ERR_UNSUPPORTED;
    }
}

void pnop_ops_free(pnop_ops* ops) { delete ops; }

int pnop_batch_submit_prepared(pnop_batch* batch, const pnop_ops* ops, const void* u0, double E0, double horizon,
                               int* id_out) {
    pnop_ctx* c = bctx(batch);
    return guarded(c, [&]() -> int {
        if (!ops) throw Status(PNOP_ERR_INVALID_ARG, "ops is NULL");
        const int id = batch_submit(c, ops->h, (const double2*)u0, E0, horizon);
        if (id_out) *id_out = id;
        return PNOP_OK;
    });
}

int pnop_batch_submit(pnop_batch* batch, const pnop_params* request, const void* u0, double E0, double horizon,
                      int* id_out) {
    pnop_ctx* c = bctx(batch);
    return guarded(c, [&]() -> int {
        const pnop::HostOps hs = batch_prepare(c, request);
        const int id = batch_submit(c, hs, (const double2*)u0, E0, horizon);
        if (id_out) *id_out = id;
        return PNOP_OK;
    });
}

int pnop_batch_run(pnop_batch* batch, int max_ticks, int* ticks_out, int* running_out) {
    pnop_ctx* c = bctx(batch);
    return guarded(c, [&]() -> int {
        if (max_ticks < 0) throw Status(PNOP_ERR_INVALID_ARG, "max_ticks must be >= 0");
        int t = 0;
        while (t < max_ticks && batch_tick(c)) ++t;
        int running = 0;
        for (const BatchReq& r : c->breq) running += (r.active && !r.done) ? 1 : 0;
        if (ticks_out) *ticks_out = t;
        if (running_out) *running_out = running;
        return PNOP_OK;
    });
}

static BatchReq* find_req(pnop_ctx* c, int id, int* slot) {
    for (int i = 0; i < c->nslot; ++i)
        if (c->breq[i].active && c->breq[i].id == id) {
            if (slot) *slot = i;
            return &c->breq[i];
        }
    throw Status(PNOP_ERR_INVALID_ARG, "no such request in the batch");
}

int pnop_batch_poll(pnop_batch* batch, int id, int* done_out) {
    pnop_ctx* c = bctx(batch);
    return guarded(c, [&]() -> int {
        BatchReq* r = find_req(c, id, nullptr);
        int done = 0;
        if (r->done) {
            const cudaError_t e = cudaEventQuery(r->ev_done);
            if (e == cudaSuccess) done = 1;
            else if (e != cudaErrorNotReady) ck(e, "poll");
        }
        if (done_out) *done_out = done;
        return PNOP_OK;
    });
}

int pnop_batch_result(pnop_batch* batch, int id, void* grad_out, double* gain_out) {
    pnop_ctx* c = bctx(batch);
    return guarded(c, [&]() -> int {
        int slot = -1;
        BatchReq* r = find_req(c, id, &slot);
        if (!r->done) throw Status(PNOP_ERR_INVALID_ARG, "request not finished: run more ticks");
        // the copies wait for this request's own completion only (not for the
        // steps of other requests queued after it): they run on the copy stream
        if (!c->copy) ck(cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking), "copy stream");
        ck(cudaStreamWaitEvent(c->copy, r->ev_done, 0), "wait request");
        double e0 = 0, eT = 0;
        ck(cudaMemcpyAsync(&e0, c->d_e0 + slot, sizeof(double), cudaMemcpyDeviceToHost, c->copy), "energy copy");
        ck(cudaMemcpyAsync(&eT, c->d_eT + slot, sizeof(double), cudaMemcpyDeviceToHost, c->copy), "energy copy");
        if (grad_out)
            ck(cudaMemcpyAsync(grad_out, slot_ptr(c, c->uN, slot), c->field_bytes(), cudaMemcpyDeviceToDevice,
                               c->copy), "gradient copy");
        ck(cudaStreamSynchronize(c->copy), "result sync");
        r->active = false;  // the slot is free again
        r->fetched = true;
        if (gain_out) *gain_out = eT / e0;
        if (!(e0 > 0) || !std::isfinite(e0)) throw Status(PNOP_ERR_NONFINITE, "initial field has no finite energy");
        if (!std::isfinite(eT)) throw Status(PNOP_ERR_NONFINITE, "final energy is not finite");
        return PNOP_OK;
    });
}

int pnop_batch_stats(const pnop_batch* batch, long long* ticks, long long* entries, long long* launches) {
    const pnop_ctx* c = bctx_c(batch);
    if (!c) return PNOP_ERR_INVALID_ARG;
    if (ticks) *ticks = c->b_ticks;
    if (entries) *entries = c->b_launch_entries;
    if (launches) {
        long long n = 0;
        for (int i = 0; i < PNOP_K_NCLASS; ++i) n += c->launches[i];
        *launches = n;
    }
    return PNOP_OK;
}

const char* pnop_batch_last_error(const pnop_batch* batch) { return pnop_last_error(bctx_c(batch)); }

void pnop_batch_destroy(pnop_batch* batch) { pnop_destroy(bctx(batch)); }

int pnop_inner(pnop_ctx* ctx, const void* a, const void* b, double* out) {
    return guarded(ctx, [&]() -> int {
        if (!a || !b || !out) throw Status(PNOP_ERR_INVALID_ARG, "bad arguments");
        *out = inner_sync(ctx, (const double2*)a, (const double2*)b);
        return PNOP_OK;
    });
}

}  // extern "C"
