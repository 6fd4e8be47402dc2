#!/usr/bin/env python
"""Throughput of the checkpointed forward+adjoint gradient on one GB300.

Workload (the metric's 64x64x256 configuration): nr=64 radial points,
|m| <= 31, 0 <= k <= 127 (96 x 384 physical, 3/2 rule), Lz = 100 radii,
Re = 2000 (mean), Wo = 8, A = 1, dt = 0.0025, start at tau0 = T/4
(deceleration, T = 2 pi Re / Wo^2), oblique m = +-1 seed (axial length 1.25
radii) plus a weak random background scaled to E0 = 1e-5.  One bench step is
one pnop_gradient over a horizon of H time steps (default 100) with a
binomial checkpoint budget of s snapshots (default 57, the slots-per-step
ratio that about 11,000 state slots in 280 GB give the 19,635-step
deceleration horizon): forward sweep, recomputation from checkpoints and H
adjoint steps.  The metric is
forward+adjoint time steps per second (H x steps / time), reported for the
mixed path (FP32 transforms and products, FP64 radial solves and inner
products) as `value`, and for the plain FP64 path under "fp64".

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the oracle is the reference arm: the method has
no other implementation to run).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# ------------------------------------------------------------------ workload
NR, NTHETA, NZ = 64, 64, 256
LZ, RE, WO, AMP, DT = 100.0, 2000.0, 8.0, 1.0, 0.0025
TAU0 = 0.25 * 2.0 * math.pi * RE / WO ** 2
E0 = 1e-5
M, K = NTHETA // 2 - 1, NZ // 2 - 1
NT, NZP = 3 * (M + 1), 3 * (K + 1)
S_VALUES = NR * (2 * M + 1) * (K + 1)
FIELD_BYTES = 3 * S_VALUES * 16
L2_BYTES = 129 * 2 ** 20

FP64_FLOPS_PER_CLK_SM = 4      # 2 FP64 FMA lanes per SM (GB300)
FP32_FLOPS_PER_CLK_SM = 256    # 128 FP32 FMA lanes per SM
N_SM = 152


def workload_name(h, s):
    return (f"checkpointed fwd+adj gradient, nr={NR} ntheta={NTHETA} nz={NZ} (|m|<={M}, |k|<={K}, {NT}x{NZP} physical),"
            f" Lz={LZ:g}, Re={RE:g}, Wo={WO:g}, A={AMP:g}, dt={DT:g}, tau0=T/4, horizon {h} steps, {s} snapshots,"
            f" oblique m=+-1 seed at E0={E0:g}")


def make_u0(r):
    from paper_2509_10103_gb300 import synth
    return synth.oblique_field(r, M, K, LZ, seed=0)


# ------------------------------------------------------------------ peaks
def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tflops(per_clk_sm, sm_max_mhz):
    return N_SM * per_clk_sm * sm_max_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ algorithmic work per unit
def fft_flops(n, real=False):
    f = 5.0 * n * math.log2(n)
    return 0.5 * f if real else f


def class_work(cls, units, mixed):
    """(flops, bytes) of `units` work units of a kernel class (algorithmic, ideal reuse)."""
    cz = 8 if mixed else 16  # complex element bytes of transform intermediates
    if cls == "synth_theta":   # one column: Nm spectral FP64 in, Nt out
        return units * fft_flops(NT), units * ((2 * M + 1) * 16 + NT * cz)
    if cls == "anal_theta":
        return units * fft_flops(NT), units * (NT * cz + (2 * M + 1) * 16)
    if cls in ("zpass_fwd", "zpass_adj"):
        nin, nout = (6, 3) if cls == "zpass_fwd" else (9, 6)
        fl = (nin + nout) * fft_flops(NZP, real=True) + (9 if cls == "zpass_fwd" else 18) * NZP
        return units * fl, units * (nin + nout) * (K + 1) * cz
    if cls in ("radial_band", "spectral"):  # the library counts algorithmic FP64 flops as units
        return units, None
    if cls == "radial_solve":
        # one banded system with a real matrix and a complex right-hand side:
        # nonzeros of the factors are 4 nr - 10 below the diagonal (4 per row,
        # fewer in rows 0..3) and 4 nr + 6 above it (8 in the wall rows 0..3,
        # 4 in the interior, fewer in the last rows), plus one scaling by the
        # inverse diagonal per row: 8 nr - 4 FMAs and nr multiplies per real part
        fl = 2.0 * (2.0 * (8 * NR - 4) + NR)
        by = NR * (13 * 8 + 2 * 16)  # factor rows (stored band) + read and write of the complex value
        return units * fl, units * by
    return None, None


KERNEL_SOURCES = ("kernels.cu", "transforms.cu", "kernels.hpp", "dev_common.cuh", "dev_df.cuh")
# the translation unit and headers that define a class's kernels: the banded
# solves live in kernels.cu, which the transforms' unit cannot change
CLASS_SOURCES = {"radial_solve": ("kernels.cu", "kernels.hpp", "dev_common.cuh", "dev_df.cuh")}


def kernel_digest(cls=None):
    """Digest of the sources of a kernel class (all kernel sources when the
    class is not listed), recorded beside every committed ncu traffic figure."""
    import hashlib
    h = hashlib.sha256()
    for f in CLASS_SOURCES.get(cls, KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_2509_10103_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_table():
    """DRAM bytes per launch from the committed ncu capture, per (class,
    precision), kept only when the capture was taken of the class's kernel
    sources as they are now (its digest matches): a figure of an older kernel
    is null."""
    out = {}
    p = os.path.join(ROOT, "profiles", "dram_traffic_per_launch.txt")
    if os.path.exists(p):
        for line in open(p):
            parts = line.split()
            if len(parts) == 5 and parts[0] == "traffic" and parts[4] == kernel_digest(parts[1]):
                out[(parts[1], parts[2])] = float(parts[3])
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = str(gpu_index)
        try:
            import torch
            u = str(torch.cuda.get_device_properties(gpu_index).uuid)
            self.idx = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip() for l in self.f.read().splitlines() if l.strip() and not l.startswith("index")]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            c = [x.strip() for x in r.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1].split()[0]))
                mx.append(float(c[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ distributed helpers
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("PNOP_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(horizon_steps, steps, ws, ms_max):
    """Whole-job fwd+adj steps/s: every rank runs its own gradients (replicas);
    the slowest rank's time bounds the job."""
    return horizon_steps * steps * ws / (ms_max / 1e3)


# ------------------------------------------------------------------ GPU arm
def time_gradient(L, torch, precision, steps, warmup, H, snaps, ws, rank, sampler=None, host_slots=0,
                  profile_pass=True):
    ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, precision, snaps)
    if host_slots:
        ctx.pnop_set_host_tier(host_slots, -1.0)  # io ratio measured on this device
    import numpy as np
    r = np.array(ctx.pnop_grid_points())
    u0 = torch.from_numpy(make_u0(r)).to("cuda")
    g = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    horizon = H * DT
    # warm-up; the first warm-up step times every kernel class to find the dominant one
    ctx.pnop_profile((1 << len(L.KCLASSES)) - 1)
    gain = ctx.pnop_gradient(u0, E0, horizon, g)
    prof = ctx.pnop_profile_read()
    for _ in range(max(0, warmup - 1)):
        gain = ctx.pnop_gradient(u0, E0, horizon, g)
    dom = max(prof, key=lambda k: prof[k][0])
    # the timed region runs with per-launch event timing off (counters only)
    ctx.pnop_profile(0)
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gain = ctx.pnop_gradient(u0, E0, horizon, g)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(ws)
    ms = e0.elapsed_time(e1)
    counts = ctx.pnop_profile_read()
    # the same steps once more with CUDA events around every launch of the
    # dominant class, on the stream each launch goes to: its average launch
    # duration for the roofline (this pass is not part of `value`)
    tprof = None
    if profile_pass:
        ctx.pnop_profile(1 << L.KCLASSES.index(dom))
        for _ in range(steps):
            ctx.pnop_gradient(u0, E0, horizon, g)
        torch.cuda.synchronize()
        tprof = ctx.pnop_profile_read()
    adv, nadj, stores = ctx.pnop_gradient_stats()
    host = ctx.pnop_host_tier_stats() if host_slots else None
    ctx.close()
    return {"ms": ms, "gain": gain, "warm_profile": prof, "timed_profile": tprof, "timed_counts": counts,
            "dominant": dom,
            "advances": adv, "adjoint_steps": nadj, "stores": stores, "clocks": clocks, "host": host}


def accuracy_vs_fp64(L, torch, H, snaps, precisions):
    """Gain relative error and gradient cosine (energy inner product) of each
    precision's gradient against the FP64 gradient on the bench workload (the
    FP64 path is pinned to the oracle by the parity tests)."""
    import numpy as np
    out, ref = {}, None
    for prec in (L.PNOP_FP64,) + tuple(precisions):
        ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, prec, snaps)
        r = np.array(ctx.pnop_grid_points())
        u0 = torch.from_numpy(make_u0(r)).to("cuda")
        g = torch.zeros_like(u0)
        gain = ctx.pnop_gradient(u0, E0, H * DT, g)
        if ref is None:
            ref = (gain, g, ctx)
            continue
        c64 = ref[2]
        cos = c64.pnop_inner(g, ref[1]) / math.sqrt(c64.pnop_inner(g, g) * c64.pnop_inner(ref[1], ref[1]))
        out[PREC_NAMES[prec]] = {"gain_rel_err_vs_fp64": abs(gain / ref[0] - 1), "gradient_cosine_vs_fp64": cos}
        ctx.close()
    ref[2].close()
    return out


PREC_NAMES = {0: "fp64", 1: "mixed", 2: "df", 3: "mixed_df"}
DTYPES = {0: "f64", 1: "f32 transforms + f64", 2: "double-f32 banded products + f64",
          3: "f32 transforms + double-f32 banded products + f64"}


def time_single_steps(L, torch, precision, reps=20):
    """Raw device time of one forward step and of one adjoint step (no checkpointing)."""
    import numpy as np
    ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, precision, 1)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(make_u0(r)).to("cuda")
    u *= math.sqrt(E0 / ctx.pnop_energy(u))
    lam = u.clone()
    x = u.clone()
    for _ in range(3):
        ctx.pnop_step_forward(x, TAU0, 1)
        ctx.pnop_step_adjoint(u, lam, TAU0)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record()
    for _ in range(reps):
        ctx.pnop_step_forward(x, TAU0, 1)
    e[1].record()
    for _ in range(reps):
        ctx.pnop_step_adjoint(u, lam, TAU0)
    e[2].record()
    torch.cuda.synchronize()
    out = {"forward_step_ms": e[0].elapsed_time(e[1]) / reps, "adjoint_step_ms": e[1].elapsed_time(e[2]) / reps}
    ctx.close()
    return out


def budget_sweep(L, torch, precision, H, budgets=(10, 57, 100), steps=2):
    """fwd+adj steps/s of the same gradient at several checkpoint budgets (recompute vs store)."""
    out = {}
    for s in budgets:
        res = time_gradient(L, torch, precision, steps, 1, H, s, 1, 0, None, profile_pass=False)
        out[str(s)] = {"steps_per_s": H * steps / (res["ms"] / 1e3), "advances": res["advances"]}
    return out


def continuous_adjoint_report(L, torch, precision, H, snaps, steps=2):
    """The gradient through the continuous adjoint (pnop_gradient_continuous) on
    the same workload, and its agreement with the exact discrete gradient
    (both projected onto admissible fields)."""
    import numpy as np
    ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, precision, snaps)
    r = np.array(ctx.pnop_grid_points())
    u0 = torch.from_numpy(make_u0(r)).to("cuda")
    gc, gd = torch.zeros_like(u0), torch.zeros_like(u0)
    horizon = H * DT
    ctx.pnop_gradient_continuous(u0, E0, horizon, gc)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ctx.pnop_gradient_continuous(u0, E0, horizon, gc)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.pnop_gradient(u0, E0, horizon, gd)
    pc, pd = torch.zeros_like(u0), torch.zeros_like(u0)
    ctx.pnop_apply(L.OP_PROJECT, gc, None, pc)
    ctx.pnop_apply(L.OP_PROJECT, gd, None, pd)
    cos = ctx.pnop_inner(pc, pd) / math.sqrt(ctx.pnop_inner(pc, pc) * ctx.pnop_inner(pd, pd))
    ctx.close()
    return {"steps_per_s": H * steps / (ms / 1e3), "snap_budget": snaps,
            "cosine_with_discrete_gradient_projected": cos}


def host_tier_report(L, torch, precision, H, snaps=10, steps=2):
    """The same gradient with `snaps` HBM checkpoint slots plus up to H - 1 pinned
    host slots (two-level schedule, Eq. 2.21, io ratio measured)."""
    res = time_gradient(L, torch, precision, steps, 1, H, snaps, 1, 0, None, host_slots=H - 1, profile_pass=False)
    return {"hbm_slots": snaps, "max_host_slots": H - 1, "steps_per_s": H * steps / (res["ms"] / 1e3),
            "advances": res["advances"], **res["host"]}


def time_e2e(L, torch, precision, steps, warmup, H, snaps):
    ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, precision, snaps)
    import numpy as np
    r = np.array(ctx.pnop_grid_points())
    u0h = torch.from_numpy(make_u0(r)).pin_memory()
    gh = torch.zeros(ctx.shape, dtype=torch.complex128).pin_memory()
    for _ in range(warmup):
        ctx.pnop_gradient_host(u0h, E0, H * DT, gh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.pnop_gradient_host(u0h, E0, H * DT, gh)
    torch.cuda.synchronize()
    s = time.perf_counter() - t0
    ctx.close()
    return s


def roofline(L, res, mixed, peaks, pk_src, alu_measured=None, prec_name=None):
    """Roofline of the dominant class.  alu_measured: {"fp64": T, "fp32": T}
    from the library's FMA probe on this device (TFLOP/s); the ALU peak is
    the measured figure when given, the derived one (SMs x lanes x clock)
    otherwise, and both are reported."""
    cls = res["dominant"]
    ms, launches, units = res["timed_profile"][cls]
    fl, by = class_work(cls, units, mixed)
    hbm = peaks.get("hbm_gbs", 6800.0)
    smx = peaks.get("sm_max_mhz", 2070.0)
    if fl is None or launches == 0 or ms <= 0:
        return None
    fp32 = mixed and cls not in ("radial_solve", "radial_band", "spectral")
    per_clk = FP32_FLOPS_PER_CLK_SM if fp32 else FP64_FLOPS_PER_CLK_SM
    derived = alu_peak_tflops(per_clk, smx)
    meas = (alu_measured or {}).get("fp32" if fp32 else "fp64")
    fp_peak = meas if meas else derived
    t = ms / 1e3
    ach_f = fl / t / 1e12
    ach_b = by / t / 1e9 if by is not None else None
    frac_f = ach_f / fp_peak
    frac_b = ach_b / hbm if by is not None else 0.0
    tt = traffic_table().get((cls, prec_name or ("mixed" if mixed else "fp64")))
    base = {"kernel": cls, "launches": launches, "avg_launch_us": ms * 1e3 / launches,
            "traffic": tt,
            "traffic_note": "ncu DRAM bytes per launch of the current kernel sources (profiles/), null when the"
                            " committed capture predates them"}
    if frac_f >= frac_b:
        src = (f"measured: {'FP32' if fp32 else 'FP64'} FMA probe pnop_measure_fma_peak on this GPU" if meas else
               f"derived: {N_SM} SMs x {per_clk} flop/clk x {smx:g} MHz")
        base.update({"bound": "alu", "achieved": ach_f, "peak": fp_peak, "unit": "TFLOP/s", "frac": frac_f,
                     "peak_source": src, "peak_derived": derived, "frac_of_derived": ach_f / derived})
        if by is not None:
            base["hbm_frac"] = frac_b
        elif tt:  # the class counts flops only: its HBM use from the measured DRAM traffic per launch
            base["hbm_frac_of_measured_traffic"] = tt / (t / launches) / 1e9 / hbm
    else:
        base.update({"bound": "hbm", "achieved": ach_b, "peak": hbm, "unit": "GB/s", "frac": frac_b,
                     "peak_source": f"{pk_src} (MEASURED_PEAKS.json hbm_gbs)" if pk_src == "measured" else "fallback",
                     "alu_frac": frac_f})
    return base


def optimise_full_report(L, torch, E0_opt=1e-5, iters=10, precision=None):
    """Adjoint looping (pnop_optimise, Section 2.3, Eq. 2.13-2.15) on the full
    nonlinear optimisation workload: the 64x64x256 grid and physics above,
    start at tau0 = T/4 (deceleration), horizon T/4 = 19,635 steps of
    dt = 0.0025, seeded oblique initial guess, mixed precision, checkpoint
    pool sized from free HBM (snap_budget 0).  Reports G per iteration and the
    seconds per gradient."""
    import numpy as np
    precision = L.PNOP_MIXED if precision is None else precision
    T = 2.0 * math.pi * RE / WO ** 2
    nsteps = int(round(0.25 * T / DT))
    ctx = L.Context(NR, NTHETA, NZ, LZ, RE, DT, WO, AMP, TAU0, precision, 0)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(make_u0(r)).to("cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats, hist = ctx.pnop_optimise(u, E0_opt, nsteps * DT, iters, 1e-8)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    adv, nadj, stores = ctx.pnop_gradient_stats()
    out = {"workload": f"nr={NR} ntheta={NTHETA} nz={NZ}, Lz={LZ:g}, Re={RE:g}, Wo={WO:g}, A={AMP:g}, tau0=T/4,"
                       f" horizon T/4 = {nsteps} steps of dt={DT:g}, oblique seed, E0={E0_opt:g}",
           "precision": "mixed" if precision == L.PNOP_MIXED else "fp64",
           "iterations": stats["iterations"], "gradients": stats["gradients"], "forward_evals": stats["forward_evals"],
           "converged": stats["converged"], "gain_history": hist, "wall_s": wall,
           # every gradient is one forward sweep (checkpoints stored) plus one adjoint sweep; rejected
           # line-search trials add forward sweeps, counted in forward_evals
           "seconds_per_gradient": wall / max(1, stats["gradients"]),
           "advances_last_sweep": adv, "adjoint_steps_last_sweep": nadj,
           "device_gb": ctx.pnop_device_bytes() / 2 ** 30}
    ctx.close()
    return out


# ------------------------------------------------------------------ serving stream
SERVE_RES = ((32, 32, 64, 10.0), (48, 48, 128, 25.0), (64, 64, 256, 50.0))


def _serving_requests(L, nreq, seed, arrivals, full=False):
    """Seeded requests: resolution from SERVE_RES, Re in [1500, 3000], A in
    [0.5, 1.5], Wo in [4, 18], E0 = 10^U(-7,-4), dt = 0.005, mixed precision.
    full: horizons of 1-10 time units (200-2000 steps), 64 checkpoint slots
    each; otherwise 10-50 steps (shortened so that the stream stays within a
    minute) and 8 slots."""
    import numpy as np
    from paper_2509_10103_gb300 import serving, synth
    rng = np.random.default_rng(seed)
    fields = {}
    for (nr, nth, nz, lz) in SERVE_RES:
        ctx = L.Context(nr, nth, nz, lz, 2000.0, 0.005, 8.0, 1.0, 0.0, L.PNOP_MIXED, 1)
        r = np.array(ctx.pnop_grid_points())
        ctx.close()
        fields[(nr, nth, nz)] = synth.random_field(r, nth // 2 - 1, nz // 2 - 1, lz, seed=seed + nr)
    reqs = []
    for i in range(nreq):
        nr, nth, nz, lz = SERVE_RES[int(rng.integers(len(SERVE_RES)))]
        n = int(rng.integers(200, 2001)) if full else int(rng.integers(10, 51))
        reqs.append(serving.Request(rid=i, nr=nr, ntheta=nth, nz=nz, Lz=lz, Re=float(rng.uniform(1500, 3000)),
                                    Wo=float(rng.uniform(4, 18)), A=float(rng.uniform(0.5, 1.5)),
                                    tau0=float(rng.uniform(0, 100)), E0=float(10 ** rng.uniform(-7, -4)),
                                    horizon=n * 0.005, dt=0.005, u0=fields[(nr, nth, nz)], precision=L.PNOP_MIXED,
                                    snaps=64 if full else 8, arrival=float(arrivals[i])))
    return reqs


def serving_report(L, nreq=256, probe=48, load=0.7, seed=0, budget=40 << 30, max_active=8, batched=False,
                   full=False):
    """Capacity probe, then a Poisson stream at `load` x that capacity.

    The probe submits `probe` requests at once and takes completed / wall as
    the capacity (requests/s).  The stream then offers `nreq` requests with
    exponential gaps of mean 1 / (load x capacity) and reports p50/p99
    latency (arrival to result on the host) and throughput.  batched: the
    BatchServer (max_active slots per batch of one resolution, more batches
    of a resolution as its requests need them, shared launches) instead of one
    context and stream per request.  full: the stated horizons of 1-10 time
    units (see _serving_requests)."""
    import numpy as np
    from paper_2509_10103_gb300 import serving
    reqs = _serving_requests(L, probe, seed + 1, np.zeros(probe), full)
    t0 = time.perf_counter()
    # both servers run at most max_active requests at once (the batched one over all its batches)
    cap_total = max_active if batched else None
    res, _ = serving.serve_stream(reqs, hbm_budget=budget, max_active=max_active, batched=batched,
                                  max_active_total=cap_total)
    cap = sum(r.error is None for r in res) / (time.perf_counter() - t0)
    rate = load * cap
    gaps = np.random.default_rng(seed + 2).exponential(1.0 / rate, nreq)
    reqs = _serving_requests(L, nreq, seed, np.cumsum(gaps), full)
    t0 = time.perf_counter()
    res, srv = serving.serve_stream(reqs, hbm_budget=budget, max_active=max_active, batched=batched,
                                    max_active_total=cap_total)
    wall = time.perf_counter() - t0
    ok = [r for r in res if r.error is None]
    steps = sum(int(round(q.horizon / q.dt)) for q, r in zip(reqs, res) if r.error is None)
    lat = serving.latency_summary(res)
    return {"requests": nreq, "completed": len(ok), "errors": [r.error for r in res if r.error][:3],
            "resolutions": [f"{a}x{b}x{c}" for a, b, c, _ in SERVE_RES], "precision": "mixed",
            "capacity_req_s": cap, "capacity_probe": f"{probe} requests submitted at once",
            "offered_load": load, "offered_rate_req_s": rate, "throughput_req_s": len(ok) / wall,
            "steps_per_s": steps / wall, "p50_latency_s": lat["p50_s"], "p99_latency_s": lat["p99_s"],
            "mean_latency_s": lat.get("mean_s"), "peak_active": srv.peak_active,
            "peak_admitted_gb": srv.peak_bytes / 2 ** 30, "hbm_budget_gb": budget / 2 ** 30, "wall_s": wall,
            "horizons": "200-2000 steps of dt=0.005 (1-10 time units), 64 checkpoint slots" if full else
                        "10-50 steps of dt=0.005, 8 checkpoint slots",
            "arrivals": f"Poisson at {load} x measured capacity",
            "server": (f"batched launches per resolution (BatchServer), at most {max_active} requests running"
                       if batched else f"one context and stream per request, at most {max_active} running"),
            "peak_requests_in_one_batch": getattr(srv, "peak_batch", None),
            "peak_batches_of_one_resolution": getattr(srv, "peak_batches_per_kind", None),
            "batches_created": getattr(srv, "batches_made", None)}


def batch_report(L, torch, nsteps=20, snaps=8, seed=7, only=None):
    """Batched gradients (pnop_batch) against the same requests one after
    another on single contexts, per serving resolution: B requests of seeded
    physics (as the serving stream), nsteps steps of dt = 0.005 each.
    Operator set-up (host) is outside both timings; the batched time runs
    from the first queued step to the last fetched gradient."""
    import numpy as np
    from paper_2509_10103_gb300 import synth
    rng = np.random.default_rng(seed)
    out = {}
    cases = [(res, L.PNOP_MIXED, 16 if res[0] < 64 else 8) for res in SERVE_RES] + [(SERVE_RES[0], L.PNOP_FP64, 16)]
    if only is not None:  # one resolution (mixed) only
        cases = [c for c in cases if c[0][:3] == tuple(only) and c[1] == L.PNOP_MIXED]
    for (nr, nth, nz, lz), prec, B in cases:
        ctx = L.Context(nr, nth, nz, lz, 2000.0, 0.005, 8.0, 1.0, 0.0, prec, 1)
        r = np.array(ctx.pnop_grid_points())
        ctx.close()
        u = torch.from_numpy(synth.random_field(r, nth // 2 - 1, nz // 2 - 1, lz, seed=seed + nr)).to("cuda")
        phys = [(float(rng.uniform(1500, 3000)), float(rng.uniform(4, 18)), float(rng.uniform(0.5, 1.5)),
                 float(rng.uniform(0, 100)), float(10 ** rng.uniform(-7, -4))) for _ in range(B)]
        H = nsteps * 0.005
        g = torch.empty_like(u)
        # batched
        b = L.Batch(nr, nth, nz, lz, B, prec, snaps)
        for rep in range(2):  # the first pass warms up
            ids = [b.pnop_batch_submit(u, E0, H, Re, 0.005, Wo, A, t0) for Re, Wo, A, t0, E0 in phys]
            torch.cuda.synchronize()
            st0 = b.pnop_batch_stats()
            t0 = time.perf_counter()
            b.pnop_batch_run(1 << 30)
            for i in ids:
                b.pnop_batch_result(i, g)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            st = b.pnop_batch_stats()
        b.close()
        # one after another on single contexts
        ctxs = [L.Context(nr, nth, nz, lz, Re, 0.005, Wo, A, t0, prec, snaps) for Re, Wo, A, t0, E0 in phys]
        ctxs[0].pnop_gradient(u, phys[0][4], H, g)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, (Re, Wo, A, tt, E0) in zip(ctxs, phys):
            c.pnop_gradient(u, E0, H, g)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        ticks = st["ticks"] - st0["ticks"]
        key = f"{nr}x{nth}x{nz}_{'mixed' if prec == L.PNOP_MIXED else 'fp64'}"
        out[key] = {"requests": B, "steps_each": nsteps, "snap_budget": snaps,
                    "batched_steps_per_s": B * nsteps / tb, "single_steps_per_s": B * nsteps / ts,
                    "speedup": ts / tb, "batched_ticks": ticks,
                    "mean_requests_per_launch": (st["entries"] - st0["entries"]) / max(1, ticks),
                    "kernel_launches_batched": st["launches"] - st0["launches"]}
    return out


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)
ORACLE_SAMPLE_CODE = r"""
import os, sys, time, json, math
sys.path.insert(0, sys.argv[1])
import numpy as np
from oracle import pipe_oracle as po
import bench as B
planes, modes = int(sys.argv[2]), int(sys.argv[3])
o = po.Oracle(po.Params(nr=B.NR, M=B.M, K=B.K, Lz=B.LZ, Re=B.RE, dt=B.DT, Wo=B.WO, A=B.AMP))
u = o.scale_to(B.make_u0(o.r), B.E0)
t = B.TAU0
T = {}
t0 = time.perf_counter(); w = o.curl(u); T['curl'] = time.perf_counter() - t0
sl = slice(0, planes)
t0 = time.perf_counter()
up = np.stack([o.synth(c[sl]) for c in u]); wp = np.stack([o.synth(c[sl]) for c in w])
n = np.stack([o.analysis(c) for c in np.cross(up, wp, axis=0)])
T['nl_planes'] = time.perf_counter() - t0
t0 = time.perf_counter()
gb = np.stack([o.analysisT(c) for c in n])
upb = np.cross(wp, gb, axis=0); wpb = np.cross(gb, up, axis=0)
ub = np.stack([o.synthT(c) for c in upb]); wb = np.stack([o.synthT(c) for c in wpb])
T['nlT_planes'] = time.perf_counter() - t0
rng = np.random.default_rng(0)
sel = [(int(rng.integers(-B.M, B.M + 1)), int(rng.integers(0, B.K + 1))) for _ in range(modes)]
t0 = time.perf_counter()
for (m, k) in sel: o.mode_maps(m, k)
T['maps_build'] = time.perf_counter() - t0
t0 = time.perf_counter()
for rep in range(10):
    for (m, k) in sel:
        Su, SF = o.mode_maps(m, k)
        v = u[:, :, m + B.M, k].reshape(-1); Su @ v + SF @ v
T['stage_apply'] = (time.perf_counter() - t0) / 10
scale_p = B.NR / planes
scale_m = (2 * B.M + 1) * (B.K + 1) / modes
nl = T['curl'] + T['nl_planes'] * scale_p
nlT = 2 * T['curl'] + T['nlT_planes'] * scale_p
st = T['stage_apply'] * scale_m
# oracle gradient per time step (store-all): forward 2 NL + 2 stages; adjoint 1 NL + 1 stage
# (re-run predictor) + 2 transposed NL + 2 transposed stages (two matvecs each)
per_step = 3 * nl + 2 * nlT + 3 * st + 2 * 2 * st
T['per_step_s'] = per_step
T['maps_build_total_s'] = T['maps_build'] * scale_m
print(json.dumps(T))
"""


def oracle_sample(planes=4, modes=16):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", ORACLE_SAMPLE_CODE, ROOT, str(planes), str(modes)],
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, timeout=900)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_sample_parallel(planes=16, modes=64, procs=None):
    """The same one-thread oracle sample in `procs` processes at once (all host
    cores by default): the sample's planes and modes are independent, so
    procs / (wall time) samples per second is the oracle's all-core rate."""
    procs = procs or os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ps = [subprocess.Popen([sys.executable, "-c", ORACLE_SAMPLE_CODE, ROOT, str(planes), str(modes)],
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env) for _ in range(procs)]
    outs = [p.communicate(timeout=1800) for p in ps]
    if any(p.returncode != 0 for p in ps):
        raise RuntimeError("parallel oracle sample failed")
    # each process times its own sample while all cores are busy
    return procs, [json.loads(o.strip().splitlines()[-1])["per_step_s"] for o, _ in outs]


def oracle_sample_desc(planes, modes):
    return (f"extrapolated from a bounded sample: "
            f"FP64 numpy oracle, 1 thread: curl + 3/2-padded transforms/products on {planes} of {NR} radial planes"
            f" (x{NR // planes}), stage maps applied on {modes} random (m,k) modes (x{(2 * M + 1) * (K + 1) // modes}),"
            f" combined as 3 N + 2 N^T + 3 S + 2 S^T per fwd+adj step (store-all sweep); map construction excluded")


def reference_main(args):
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    planes, modes = 8, 32
    for _ in range(args.warmup):
        oracle_sample(planes, modes)
    ts = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts.append(oracle_sample(planes, modes)["per_step_s"])
    wall = time.perf_counter() - t0
    per = statistics.median(ts)
    val = 1.0 / per
    line = {"impl": "reference", "metric": "fwd+adj steps/s at 64x64x256, mixed vs FP64 on 1 GB300; serving p50/p99 latency", "value": val, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.horizon_steps, args.snaps), "sample": "bounded oracle sample"},
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": oracle_sample_desc(planes, modes)},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--horizon-steps", type=int, default=100)
    ap.add_argument("--snaps", type=int, default=57,
                    help="checkpoint slots; 57 per 100 steps is the slots-per-step ratio of the 19,635-step "
                         "deceleration horizon when ~11,000 state slots fill 280 GB of HBM")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single-step timings and the budget sweep (profiling runs)")
    ap.add_argument("--precision", default="both", choices=["both", "mixed_df", "mixed", "fp64"],
                    help="which path(s) to time: 'both' times the mixed path with double-FP32 banded products as the"
                         " main line and the FP64 and plain mixed paths beside it; the others time one path")
    ap.add_argument("--optimise-full", action="store_true",
                    help="print only the adjoint-looping run on the full deceleration horizon (19,635 steps)")
    ap.add_argument("--opt-iters", type=int, default=10)
    ap.add_argument("--serving-full", action="store_true",
                    help="print only the serving reports (both servers) at the stated horizons of 1-10 time units")
    ap.add_argument("--only-batched", default=None, metavar="RES",
                    help="print only the batched-gradient comparison at one serving resolution (e.g. 32x32x64)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2509_10103_gb300 import build
    if rank == 0:
        build.build()
    barrier(ws)
    from paper_2509_10103_gb300 import _lib as L

    if args.optimise_full:
        print(json.dumps({"optimise_full": optimise_full_report(L, torch, iters=args.opt_iters)}))
        return 0
    if args.serving_full:
        out = {"serving_full": serving_report(L, probe=32, budget=160 << 30, full=True),
               "serving_full_batched": serving_report(L, probe=32, budget=160 << 30, batched=True, full=True)}
        print(json.dumps(out))
        return 0
    if args.only_batched:
        res = tuple(int(x) for x in args.only_batched.split("x"))
        print(json.dumps(batch_report(L, torch, only=res)))
        return 0
    peaks, pk_src = load_peaks()
    alu = {"fp64": L.pnop_measure_fma_peak(L.PNOP_FP64, 0.05), "fp32": L.pnop_measure_fma_peak(L.PNOP_MIXED, 0.05)}
    H, s = args.horizon_steps, args.snaps
    sampler = ClockSampler(local) if rank == 0 else None
    if args.precision == "fp64":
        args.no_fp64 = True
    # the main line: the mixed-precision path (FP32 transforms and products,
    # double-FP32 banded products, FP64 solves, corrections and inner
    # products) unless one path is asked for; the others are reported beside it
    main_prec = {"both": L.PNOP_MIXED_DF, "mixed_df": L.PNOP_MIXED_DF, "mixed": L.PNOP_MIXED,
                 "fp64": L.PNOP_FP64}[args.precision]
    mix = time_gradient(L, torch, main_prec, args.steps, args.warmup, H, s, ws, rank, sampler)
    ms = max_over_ranks(mix["ms"], ws)
    value = aggregate_value(H, args.steps, ws, ms)

    def side_path(prec):
        f = time_gradient(L, torch, prec, args.steps, args.warmup, H, s, ws, rank, None)
        fms = max_over_ranks(f["ms"], ws)
        return {"value": H * args.steps * ws / (fms / 1e3), "unit": "steps/s", "ms_per_step": fms / args.steps,
                "gain": f["gain"], "dtype": DTYPES[prec],
                "roofline": roofline(L, f, (prec & L.PNOP_MIXED) != 0, peaks, pk_src, alu, PREC_NAMES[prec]),
                "kernels_ms_per_step": {k: v[0] for k, v in f["warm_profile"].items()}}

    fp64 = side_path(L.PNOP_FP64) if (not args.no_fp64 and args.precision == "both") else None
    mixed_plain = side_path(L.PNOP_MIXED) if args.precision == "both" else None
    e2e_s = time_e2e(L, torch, main_prec, args.steps, args.warmup, H, s)
    e2e_s = max_over_ranks(e2e_s, ws)
    if rank != 0:
        return 0
    launches = sum(v[1] for v in mix["timed_counts"].values())
    out = {
        "metric": "fwd+adj steps/s at 64x64x256, mixed vs FP64 on 1 GB300; serving p50/p99 latency",
        "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[main_prec], "precision": PREC_NAMES[main_prec], "data": "synthetic",
        "config": {"workload": workload_name(H, s), "horizon_steps": H, "snap_budget": s,
                   "advances_per_gradient": mix["advances"], "adjoint_steps_per_gradient": mix["adjoint_steps"],
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": f"inputs and working set > L2 (state {FIELD_BYTES / 2**20:.1f} MiB x >20 buffers + transform"
                         " scratch); no flush"},
        "gain": mix["gain"],
        "roofline": roofline(L, mix, (main_prec & L.PNOP_MIXED) != 0, peaks, pk_src, alu, PREC_NAMES[main_prec]),
        "alu_peaks_measured_tflops": alu,
        "kernels_ms_per_step": {k: v[0] for k, v in mix["warm_profile"].items()},
        "fp64": fp64,
        "speedup_mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
        "mixed_fp64_banded": mixed_plain,
        "speedup_mixed_fp64_banded_over_fp64": (mixed_plain["value"] / fp64["value"]) if (fp64 and mixed_plain) else None,
        "e2e": {"value": H * args.steps * ws / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": FIELD_BYTES,
                "d2h_bytes_per_step": FIELD_BYTES + 24},
        "gpu_launches": launches,
        "clocks": mix["clocks"],
    }

    def extra(key, fn):
        """A secondary report: its failure is recorded under its key and never costs the main line."""
        try:
            out[key] = fn()
        except Exception as e:  # noqa: BLE001 - reported in the JSON line
            out[key] = {"error": f"{type(e).__name__}: {e}"[:500]}

    if ws == 1 and not args.no_extras:
        extra("accuracy", lambda: accuracy_vs_fp64(L, torch, H, s, (L.PNOP_MIXED, L.PNOP_MIXED_DF, L.PNOP_DF)))
        extra("single_step", lambda: {"mixed": time_single_steps(L, torch, L.PNOP_MIXED),
                                      "mixed_df": time_single_steps(L, torch, L.PNOP_MIXED_DF),
                                      "fp64": time_single_steps(L, torch, L.PNOP_FP64)})
        # the side reports run the main line's path
        extra("budget_sweep", lambda: budget_sweep(L, torch, main_prec, H))
        extra("host_tier", lambda: host_tier_report(L, torch, main_prec, H))
        extra("continuous_adjoint", lambda: continuous_adjoint_report(L, torch, main_prec, H, s))
        extra("batched_gradients", lambda: batch_report(L, torch))
    if not args.no_serving and ws == 1:
        extra("serving", lambda: serving_report(L))
        extra("serving_batched", lambda: serving_report(L, batched=True))
    if not args.no_cpu_baseline and ws == 1:
        planes, modes = 16, 64

        def one_core():
            smp = oracle_sample(planes, modes)
            return {"value": 1.0 / smp["per_step_s"], "unit": "steps/s", "cores": 1, "kind": "oracle",
                    "sample": oracle_sample_desc(planes, modes)}

        def all_cores():
            procs, per_step = oracle_sample_parallel(planes, modes)
            # every process extrapolates one step from its share of the cores
            return {"value": sum(1.0 / x for x in per_step), "unit": "steps/s", "cores": procs, "kind": "oracle",
                    "sample": oracle_sample_desc(planes, modes) + f"; {procs} such samples at once, one per core"}

        extra("cpu_baseline", one_core)
        if not args.no_extras:
            extra("cpu_baseline_all_cores", all_cores)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
