"""ctypes binding of libpnop (argument marshalling only).

The names mirror the C ABI in include/pnop.h.  Field arguments may be torch
tensors (complex128, contiguous, shape [3, nr, 2M+1, K+1], on the context's
device) or raw integer device pointers.  There is no fallback: if the shared
library is missing the import fails.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_longlong, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpnop.so")

PNOP_OK = 0
PNOP_FP64 = 0
PNOP_MIXED = 1      # FP32 transforms and products
PNOP_DF = 2         # double-FP32 explicit banded products
PNOP_MIXED_DF = 3
KCLASSES = ("synth_theta", "zpass_fwd", "zpass_adj", "anal_theta", "spectral", "radial_band", "radial_solve",
            "elementwise", "reduce")
OP_CURL, OP_NONLINEAR, OP_STAGE, OP_NONLINEAR_T, OP_STAGE_T_U, OP_STAGE_T_F, OP_PROJECT, OP_NONLINEAR_ADJ = range(8)

EXPORTS = (
    "pnop_create", "pnop_set_base_flow", "pnop_dims", "pnop_grid_points", "pnop_step_forward", "pnop_step_adjoint",
    "pnop_gradient", "pnop_gradient_continuous", "pnop_gradient_forward", "pnop_gradient_backward",
    "pnop_gradient_host", "pnop_gradient_stats", "pnop_optimise", "pnop_optimise_ex", "pnop_set_host_tier", "pnop_host_tier_stats",
    "pnop_two_level_counts", "pnop_mode_energy", "pnop_resolution", "pnop_energy", "pnop_inner", "pnop_apply", "pnop_set_timeout", "pnop_set_optimiser_first_step",
    "pnop_sync", "pnop_profile", "pnop_profile_read", "pnop_revolve_counts", "pnop_context_bytes", "pnop_device_bytes",
    "pnop_energy_noalloc", "pnop_measure_fma_peak", "pnop_last_error", "pnop_error_string", "pnop_destroy",
    "pnop_batch_create", "pnop_batch_submit", "pnop_batch_run", "pnop_batch_poll", "pnop_batch_result",
    "pnop_batch_stats", "pnop_batch_last_error", "pnop_batch_destroy", "pnop_batch_prepare",
    "pnop_batch_submit_prepared", "pnop_ops_free", "pnop_batch_bytes",
)


class pnop_grid(ctypes.Structure):
    _fields_ = [("nr", c_int), ("ntheta", c_int), ("nz", c_int), ("Lz", c_double), ("stretch", c_double)]


class pnop_params(ctypes.Structure):
    _fields_ = [("Re", c_double), ("Wo", c_double), ("A", c_double), ("dt", c_double), ("tau0", c_double),
                ("precision", c_int), ("snap_budget", c_int), ("hbm_budget", c_size_t)]


class pnop_opt_stats(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("gradients", c_int), ("forward_evals", c_int), ("converged", c_int),
                ("gain", c_double), ("rel_change", c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpnop.so is not built ({LIB_PATH}); run paper_2509_10103_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "pnop_create": (c_int, [POINTER(pnop_grid), POINTER(pnop_params), c_void_p, POINTER(c_void_p)]),
        "pnop_set_base_flow": (c_int, [c_void_p, c_double, c_double, c_double, c_double]),
        "pnop_dims": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
        "pnop_grid_points": (c_int, [c_void_p, POINTER(c_double)]),
        "pnop_step_forward": (c_int, [c_void_p, c_void_p, c_double, c_int]),
        "pnop_step_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_double]),
        "pnop_gradient": (c_int, [c_void_p, c_void_p, c_double, c_double, c_void_p, POINTER(c_double)]),
        "pnop_gradient_continuous": (c_int, [c_void_p, c_void_p, c_double, c_double, c_void_p, POINTER(c_double)]),
        "pnop_gradient_forward": (c_int, [c_void_p, c_void_p, c_double, c_double, POINTER(c_double), POINTER(c_double)]),
        "pnop_gradient_backward": (c_int, [c_void_p, c_double, c_int, c_void_p]),
        "pnop_gradient_host": (c_int, [c_void_p, c_void_p, c_double, c_double, c_void_p, POINTER(c_double)]),
        "pnop_gradient_stats": (c_int, [c_void_p, POINTER(c_longlong), POINTER(c_longlong), POINTER(c_longlong)]),
        "pnop_optimise": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_double, POINTER(c_double),
                                  POINTER(pnop_opt_stats)]),
        "pnop_optimise_ex": (c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_double, c_int,
                                     POINTER(c_double), POINTER(pnop_opt_stats)]),
        "pnop_set_host_tier": (c_int, [c_void_p, c_longlong, c_double]),
        "pnop_mode_energy": (c_int, [c_void_p, c_void_p, POINTER(c_double)]),
        "pnop_resolution": (c_int, [c_void_p, c_void_p, c_double, POINTER(c_double), POINTER(c_double)]),
        "pnop_host_tier_stats": (c_int, [c_void_p, POINTER(c_int), POINTER(c_longlong), POINTER(c_longlong),
                                         POINTER(c_double)]),
        "pnop_two_level_counts": (c_int, [c_longlong, c_int, c_longlong, c_double, POINTER(c_int),
                                          POINTER(c_longlong)]),
        "pnop_energy": (c_int, [c_void_p, c_void_p, POINTER(c_double)]),
        "pnop_inner": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
        "pnop_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_double]),
        "pnop_set_timeout": (c_int, [c_void_p, c_double]),
        "pnop_set_optimiser_first_step": (c_int, [c_void_p, c_double]),
        "pnop_sync": (c_int, [c_void_p]),
        "pnop_profile": (c_int, [c_void_p, ctypes.c_uint]),
        "pnop_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_longlong), POINTER(c_double)]),
        "pnop_context_bytes": (c_int, [POINTER(pnop_grid), POINTER(pnop_params), c_int, POINTER(c_size_t)]),
        "pnop_revolve_counts": (c_int, [c_int, c_int, POINTER(c_longlong), POINTER(c_longlong)]),
        "pnop_device_bytes": (c_int, [c_void_p, POINTER(c_size_t)]),
        "pnop_energy_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_double, POINTER(c_double),
                                        c_void_p]),
        "pnop_measure_fma_peak": (c_int, [c_int, c_double, c_void_p, POINTER(c_double)]),
        "pnop_last_error": (c_char_p, [c_void_p]),
        "pnop_error_string": (c_char_p, [c_int]),
        "pnop_destroy": (None, [c_void_p]),
        "pnop_batch_create": (c_int, [POINTER(pnop_grid), POINTER(pnop_params), c_int, c_void_p, POINTER(c_void_p)]),
        "pnop_batch_submit": (c_int, [c_void_p, POINTER(pnop_params), c_void_p, c_double, c_double, POINTER(c_int)]),
        "pnop_batch_run": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int)]),
        "pnop_batch_poll": (c_int, [c_void_p, c_int, POINTER(c_int)]),
        "pnop_batch_result": (c_int, [c_void_p, c_int, c_void_p, POINTER(c_double)]),
        "pnop_batch_stats": (c_int, [c_void_p, POINTER(c_longlong), POINTER(c_longlong), POINTER(c_longlong)]),
        "pnop_batch_last_error": (c_char_p, [c_void_p]),
        "pnop_batch_destroy": (None, [c_void_p]),
        "pnop_batch_prepare": (c_int, [c_void_p, POINTER(pnop_params), POINTER(c_void_p)]),
        "pnop_batch_submit_prepared": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, POINTER(c_int)]),
        "pnop_ops_free": (None, [c_void_p]),
        "pnop_batch_bytes": (c_int, [POINTER(pnop_grid), POINTER(pnop_params), c_int, POINTER(c_size_t)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class PnopError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{lib.pnop_error_string(code).decode()} ({code}): {msg}")
        self.code = code


def _ptr(x) -> int:
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("field tensors must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a torch tensor or an integer pointer")


def pnop_revolve_counts(nsteps: int, snaps: int):
    a, s = c_longlong(), c_longlong()
    rc = lib.pnop_revolve_counts(nsteps, snaps, byref(a), byref(s))
    if rc != PNOP_OK:
        raise PnopError(rc, "revolve_counts")
    return a.value, s.value


def pnop_two_level_counts(nsteps, snaps, max_host_slots, io_ratio):
    """(host checkpoints, forward steps) of the two-level schedule (host only)."""
    nf, adv = c_int(), c_longlong()
    rc = lib.pnop_two_level_counts(nsteps, snaps, max_host_slots, io_ratio, byref(nf), byref(adv))
    if rc != PNOP_OK:
        raise PnopError(rc, "two_level_counts")
    return nf.value, adv.value


def pnop_context_bytes(nr, ntheta, nz, Lz, precision, snaps):
    """Upper estimate of the device bytes of a context (host only)."""
    g = pnop_grid(nr, ntheta, nz, Lz, 0.0)
    p = pnop_params(1.0, 1.0, 0.0, 1.0, 0.0, precision, snaps, 0)
    out = c_size_t()
    rc = lib.pnop_context_bytes(byref(g), byref(p), snaps, byref(out))
    if rc != PNOP_OK:
        raise PnopError(rc, "context_bytes")
    return out.value


def pnop_batch_bytes(nr, ntheta, nz, Lz, precision, snaps, capacity):
    """Upper estimate of the device bytes of a batch (host only)."""
    g = pnop_grid(nr, ntheta, nz, Lz, 0.0)
    p = pnop_params(1.0, 1.0, 0.0, 1.0, 0.0, precision, snaps, 0)
    out = c_size_t()
    rc = lib.pnop_batch_bytes(byref(g), byref(p), capacity, byref(out))
    if rc != PNOP_OK:
        raise PnopError(rc, "batch_bytes")
    return out.value


def pnop_energy_noalloc(u, W, nr, M, K, Lz, stream=0):
    """Energy (1/2)<u,u> of a device field with no device allocation and no context.

    W: device array of the nr radial quadrature weights.  The library's scratch
    for this call is a fixed device array shared by all calls (see pnop.h)."""
    e = c_double()
    rc = lib.pnop_energy_noalloc(c_void_p(_ptr(u)), c_void_p(_ptr(W)), nr, M, K, Lz, byref(e), c_void_p(stream))
    if rc != PNOP_OK:
        raise PnopError(rc, "energy_noalloc")
    return e.value


def pnop_measure_fma_peak(precision=PNOP_FP64, seconds=0.05, stream=0):
    """Measured FMA throughput (TFLOP/s) of the current device, FP64 or FP32."""
    t = c_double()
    rc = lib.pnop_measure_fma_peak(precision, seconds, c_void_p(stream), byref(t))
    if rc != PNOP_OK:
        raise PnopError(rc, "measure_fma_peak")
    return t.value


class Context:
    """One solver context (pnop_ctx) on the current CUDA device and a stream."""

    def __init__(self, nr, ntheta, nz, Lz, Re, dt, Wo=8.0, A=1.0, tau0=0.0, precision=PNOP_FP64,
                 snap_budget=8, hbm_budget=0, stretch=0.0, stream=0):
        g = pnop_grid(nr, ntheta, nz, Lz, stretch)
        p = pnop_params(Re, Wo, A, dt, tau0, precision, snap_budget, hbm_budget)
        h = c_void_p()
        rc = lib.pnop_create(byref(g), byref(p), c_void_p(stream), byref(h))
        if rc != PNOP_OK:
            raise PnopError(rc, "pnop_create")
        self._h = h
        nr_, M, K = c_int(), c_int(), c_int()
        lib.pnop_dims(h, byref(nr_), byref(M), byref(K))
        self.nr, self.M, self.K = nr_.value, M.value, K.value
        self.Lz, self.dt, self.Re = Lz, dt, Re
        self.shape = (3, self.nr, 2 * self.M + 1, self.K + 1)

    def _check(self, rc, what):
        if rc != PNOP_OK:
            raise PnopError(rc, f"{what}: {lib.pnop_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            lib.pnop_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def pnop_grid_points(self):
        buf = (c_double * self.nr)()
        self._check(lib.pnop_grid_points(self._h, buf), "grid_points")
        return list(buf)

    def pnop_set_base_flow(self, Re, Wo, A, tau0):
        self._check(lib.pnop_set_base_flow(self._h, Re, Wo, A, tau0), "set_base_flow")
        self.Re = Re

    def pnop_step_forward(self, u, t, nsteps=1):
        self._check(lib.pnop_step_forward(self._h, c_void_p(_ptr(u)), t, nsteps), "step_forward")

    def pnop_step_adjoint(self, u_n, lam, t_n):
        self._check(lib.pnop_step_adjoint(self._h, c_void_p(_ptr(u_n)), c_void_p(_ptr(lam)), t_n), "step_adjoint")

    def pnop_gradient(self, u0, E0, horizon, grad_out):
        gain = c_double()
        self._check(lib.pnop_gradient(self._h, c_void_p(_ptr(u0)), E0, horizon, c_void_p(_ptr(grad_out)),
                                      byref(gain)), "gradient")
        return gain.value

    def pnop_gradient_continuous(self, u0, E0, horizon, grad_out):
        gain = c_double()
        self._check(lib.pnop_gradient_continuous(self._h, c_void_p(_ptr(u0)), E0, horizon,
                                                 c_void_p(_ptr(grad_out)), byref(gain)), "gradient_continuous")
        return gain.value

    def pnop_gradient_forward(self, u0, E0, horizon):
        """Forward half: returns (E(T), initial energy); checkpoints stay in the context."""
        et, e0 = c_double(), c_double()
        self._check(lib.pnop_gradient_forward(self._h, c_void_p(_ptr(u0)), E0, horizon, byref(et), byref(e0)),
                    "gradient_forward")
        return et.value, e0.value

    def pnop_gradient_backward(self, gE, grad_out, euclidean=False):
        self._check(lib.pnop_gradient_backward(self._h, gE, int(bool(euclidean)), c_void_p(_ptr(grad_out))),
                    "gradient_backward")

    def pnop_gradient_host(self, u0_host, E0, horizon, grad_host):
        """u0_host, grad_host: host arrays (numpy complex128 or pinned torch tensors)."""
        def hp(a):
            if hasattr(a, "ctypes"):
                return a.ctypes.data
            return _ptr(a)
        gain = c_double()
        self._check(lib.pnop_gradient_host(self._h, c_void_p(hp(u0_host)), E0, horizon, c_void_p(hp(grad_host)),
                                           byref(gain)), "gradient_host")
        return gain.value

    def pnop_gradient_stats(self):
        a, b, c = c_longlong(), c_longlong(), c_longlong()
        self._check(lib.pnop_gradient_stats(self._h, byref(a), byref(b), byref(c)), "gradient_stats")
        return a.value, b.value, c.value

    def pnop_optimise(self, u0, E0, horizon, max_iter, tol=1e-8, continuous=False):
        """Adjoint looping on u0 (device, in/out); returns (stats dict, gain history list).
        continuous selects the continuous adjoint for the gradients."""
        hist = (c_double * (max_iter + 1))()
        st = pnop_opt_stats()
        self._check(lib.pnop_optimise_ex(self._h, c_void_p(_ptr(u0)), E0, horizon, max_iter, tol, int(bool(continuous)),
                                         hist, byref(st)), "optimise")
        stats = {name: getattr(st, name) for name, _ in pnop_opt_stats._fields_}
        return stats, list(hist[: st.iterations + 1])

    def pnop_mode_energy(self, u):
        """Per-mode energy, shape (2, 2M+1, K+1): cross-section and axial parts."""
        import numpy as np
        nm, nk = self.shape[2], self.shape[3]
        out = np.zeros((2, nm, nk), np.float64)
        self._check(lib.pnop_mode_energy(self._h, c_void_p(_ptr(u)), out.ctypes.data_as(POINTER(c_double))),
                    "mode_energy")
        return out

    def pnop_device_bytes(self):
        """Device bytes the context holds now (checkpoint slots included)."""
        b = c_size_t()
        self._check(lib.pnop_device_bytes(self._h, byref(b)), "device_bytes")
        return b.value

    def pnop_resolution(self, u, E0=-1.0):
        """(e_M, e_K): energy of the highest azimuthal / axial mode over E0 (E0 <= 0: the field's energy)."""
        a, b = c_double(), c_double()
        self._check(lib.pnop_resolution(self._h, c_void_p(_ptr(u)), E0, byref(a), byref(b)), "resolution")
        return a.value, b.value

    def pnop_set_host_tier(self, max_host_slots, io_ratio=-1.0):
        self._check(lib.pnop_set_host_tier(self._h, max_host_slots, io_ratio), "set_host_tier")

    def pnop_host_tier_stats(self):
        nf, st, ld, r = c_int(), c_longlong(), c_longlong(), c_double()
        self._check(lib.pnop_host_tier_stats(self._h, byref(nf), byref(st), byref(ld), byref(r)), "host_tier_stats")
        return {"host_checkpoints": nf.value, "host_stores": st.value, "host_loads": ld.value, "io_ratio": r.value}

    def pnop_apply(self, op, a, b, out, t=0.0):
        bp = c_void_p(_ptr(b)) if b is not None else c_void_p(0)
        self._check(lib.pnop_apply(self._h, op, c_void_p(_ptr(a)), bp, c_void_p(_ptr(out)), t), "apply")

    def pnop_set_optimiser_first_step(self, alpha_frac):
        """First line-search step of pnop_optimise as a fraction of alpha_max (1: the paper's)."""
        self._check(lib.pnop_set_optimiser_first_step(self._h, alpha_frac), "set_optimiser_first_step")

    def pnop_set_timeout(self, seconds):
        self._check(lib.pnop_set_timeout(self._h, seconds), "set_timeout")

    def pnop_sync(self):
        self._check(lib.pnop_sync(self._h), "sync")

    def pnop_profile(self, class_mask=0):
        self._check(lib.pnop_profile(self._h, class_mask), "profile")

    def pnop_profile_read(self):
        n = len(KCLASSES)
        ms, la, un = (c_double * n)(), (c_longlong * n)(), (c_double * n)()
        self._check(lib.pnop_profile_read(self._h, ms, la, un), "profile_read")
        return {k: (ms[i], la[i], un[i]) for i, k in enumerate(KCLASSES)}

    def pnop_energy(self, u):
        e = c_double()
        self._check(lib.pnop_energy(self._h, c_void_p(_ptr(u)), byref(e)), "energy")
        return e.value

    def pnop_inner(self, a, b):
        e = c_double()
        self._check(lib.pnop_inner(self._h, c_void_p(_ptr(a)), c_void_p(_ptr(b)), byref(e)), "inner")
        return e.value


PNOP_MAX_BATCH = 16


class Batch:
    """Batched gradients of up to `capacity` requests of one grid (pnop_batch):
    one kernel launch per step kind covers every request taking that step."""

    def __init__(self, nr, ntheta, nz, Lz, capacity, precision=PNOP_FP64, snap_budget=8, hbm_budget=0,
                 stretch=0.0, stream=0):
        g = pnop_grid(nr, ntheta, nz, Lz, stretch)
        p = pnop_params(2000.0, 8.0, 1.0, 0.01, 0.0, precision, snap_budget, hbm_budget)
        h = c_void_p()
        rc = lib.pnop_batch_create(byref(g), byref(p), capacity, c_void_p(stream), byref(h))
        if rc != PNOP_OK:
            raise PnopError(rc, "pnop_batch_create")
        self._h = h
        self.capacity = capacity
        self.M, self.K = ntheta // 2 - 1, nz // 2 - 1
        self.shape = (3, nr, 2 * self.M + 1, self.K + 1)

    def _check(self, rc, what):
        if rc != PNOP_OK:
            raise PnopError(rc, f"{what}: {lib.pnop_batch_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            lib.pnop_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def pnop_batch_submit(self, u0, E0, horizon, Re, dt, Wo=8.0, A=1.0, tau0=0.0):
        """Admit one request; returns its id (u0 is copied in stream order)."""
        p = pnop_params(Re, Wo, A, dt, tau0, 0, 0, 0)
        i = c_int()
        self._check(lib.pnop_batch_submit(self._h, byref(p), c_void_p(_ptr(u0)), E0, horizon, byref(i)), "submit")
        return i.value

    def pnop_batch_prepare(self, Re, dt, Wo=8.0, A=1.0, tau0=0.0):
        """Host operators of one request (thread-safe; see pnop.h).  Returns an
        opaque handle for pnop_batch_submit_prepared; free it with pnop_ops_free."""
        p = pnop_params(Re, Wo, A, dt, tau0, 0, 0, 0)
        o = c_void_p()
        rc = lib.pnop_batch_prepare(self._h, byref(p), byref(o))
        if rc != PNOP_OK:
            raise PnopError(rc, "prepare")
        return o

    def pnop_batch_submit_prepared(self, ops, u0, E0, horizon):
        i = c_int()
        self._check(lib.pnop_batch_submit_prepared(self._h, ops, c_void_p(_ptr(u0)), E0, horizon, byref(i)),
                    "submit_prepared")
        return i.value

    @staticmethod
    def pnop_ops_free(ops):
        lib.pnop_ops_free(ops)

    def pnop_batch_run(self, max_ticks):
        """Queue up to max_ticks batched steps; returns (ticks, requests still running)."""
        t, r = c_int(), c_int()
        self._check(lib.pnop_batch_run(self._h, max_ticks, byref(t), byref(r)), "run")
        return t.value, r.value

    def pnop_batch_poll(self, rid):
        d = c_int()
        self._check(lib.pnop_batch_poll(self._h, rid, byref(d)), "poll")
        return bool(d.value)

    def pnop_batch_result(self, rid, grad_out=None):
        """(gain) of a finished request; its gradient into grad_out (device) when given."""
        gain = c_double()
        self._check(lib.pnop_batch_result(self._h, rid, c_void_p(_ptr(grad_out)) if grad_out is not None else None,
                                          byref(gain)), "result")
        return gain.value

    def pnop_batch_stats(self):
        t, e, la = c_longlong(), c_longlong(), c_longlong()
        self._check(lib.pnop_batch_stats(self._h, byref(t), byref(e), byref(la)), "stats")
        return {"ticks": t.value, "entries": e.value, "launches": la.value}
