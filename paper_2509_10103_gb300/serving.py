"""Continuous-batching servers for gradient requests of mixed parameters.

A request asks for the checkpointed gradient dE(T)/du0 and the gain G of one
initial perturbation (Eq. 2.1, 2.8, 2.12) at its own (Re, Wo, A, tau0, E0,
horizon) and resolution.  The server keeps an HBM budget: a request is
admitted as soon as a slot and its device memory (pnop_context_bytes of its
grid, precision and checkpoint slots) are free, so requests that arrive while
others run join the device work without waiting for a batch to drain.  Each
admitted request owns a context (its operators, fields and checkpoints stay on
the device until it completes) and a CUDA stream; its host thread drives the
library (ctypes releases the GIL), so kernels of different requests overlap on
the GPU.  Each request's arithmetic is independent of the others and
deterministic, so its result is the same alone and in the mix.

BatchServer goes further: requests of one grid share a pnop_batch, so each
kernel of a step is launched once for all of them (see its docstring).

The library has no counterpart in the paper: this is the serving layer named
in the workload list (continuous batching, HBM admission, p50/p99 latency).
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import _lib


@dataclass
class Request:
    rid: int
    nr: int
    ntheta: int
    nz: int
    Lz: float
    Re: float
    Wo: float
    A: float
    tau0: float
    E0: float
    horizon: float
    dt: float
    u0: np.ndarray                       # host complex128, layout of include/pnop.h
    precision: int = _lib.PNOP_MIXED
    snaps: int = 8
    arrival: float = 0.0                 # seconds after the server start
    kind: str = "gradient"               # "gradient", or "optimise": adjoint looping (Section 2.3) from u0
    max_iter: int = 10                   # optimise: iterations at most
    tol: float = 1e-8                    # optimise: relative change of G that stops the loop
    deadline: Optional[float] = None     # seconds after arrival by which it must be admitted, else dropped


@dataclass
class Result:
    """gain: G = E(T)/E0 (for "optimise", G of the optimum found); grad: the
    gradient (for "optimise", the optimised initial perturbation, energy E0);
    history: the gains of the accepted iterates ("optimise" only)."""
    rid: int
    gain: float
    grad: np.ndarray
    arrival: float
    admitted: float
    done: float
    device_bytes: int
    error: Optional[str] = None
    history: Optional[list] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


CANCELLED = "cancelled"
EXPIRED = "deadline exceeded before admission"


class Server:
    """Admits requests by HBM budget and slot count; runs each on its own stream.

    cancel(rid) drops a queued request at once; a running one finishes its
    device work (launched kernels are never interrupted) and its result is
    discarded.  A request with a deadline that is still queued when it passes
    is dropped.  Both are reported as the request's error."""

    def __init__(self, hbm_budget: int, max_active: int = 8, device: int = 0, runner=None, sizer=None):
        """runner(request, budget_bytes) -> (gain, grad) replaces the GPU runner
        and sizer(request) -> bytes the library estimate (host-side tests)."""
        self.runner = runner or self._gpu_runner
        self.sizer = sizer
        self.hbm_budget = int(hbm_budget)
        self.max_active = max_active
        self.device = device
        self.queue: deque = deque()
        self.results: dict = {}
        self.active = 0
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.peak_active = 0
        self.lock = threading.Condition()
        self.t0 = time.perf_counter()
        self.threads = []
        self.cancelled: set = set()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _drop_locked(self, r: Request, why: str) -> None:
        self.results[r.rid] = Result(r.rid, float("nan"), None, r.arrival, float("nan"), self.now(), 0, why)
        self.lock.notify_all()

    def cancel(self, rid: int) -> bool:
        """Cancel a queued or running request; False when it is unknown or done."""
        with self.lock:
            for i, (r, _) in enumerate(self.queue):
                if r.rid == rid:
                    del self.queue[i]
                    self._drop_locked(r, CANCELLED)
                    return True
            if rid in self.results:
                return False
            self.cancelled.add(rid)
            return True

    def _expire_locked(self) -> None:
        now = self.now()
        for r, need in [q for q in self.queue if q[0].deadline is not None and now - q[0].arrival > q[0].deadline]:
            self.queue.remove((r, need))
            self._drop_locked(r, EXPIRED)

    def request_bytes(self, r: Request) -> int:
        if self.sizer is not None:
            return int(self.sizer(r))
        return _lib.pnop_context_bytes(r.nr, r.ntheta, r.nz, r.Lz, r.precision, r.snaps)

    def submit(self, r: Request) -> None:
        need = self.request_bytes(r)
        if need > self.hbm_budget:
            raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
        with self.lock:
            self.queue.append((r, need))
            self._admit_locked()

    def _admit_locked(self) -> None:
        self._expire_locked()
        # first come, first served: the head waits until its memory fits
        while self.queue and self.active < self.max_active:
            r, need = self.queue[0]
            if self.bytes_in_use + need > self.hbm_budget:
                break
            self.queue.popleft()
            self.active += 1
            self.bytes_in_use += need
            self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
            self.peak_active = max(self.peak_active, self.active)
            t = threading.Thread(target=self._run, args=(r, need, self.now()), daemon=True)
            self.threads.append(t)
            t.start()

    def _gpu_runner(self, r: Request, need: int):
        import torch

        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        ctx = _lib.Context(r.nr, r.ntheta, r.nz, r.Lz, r.Re, r.dt, r.Wo, r.A, r.tau0, r.precision, r.snaps,
                           hbm_budget=need, stream=stream.cuda_stream)
        try:
            dev = f"cuda:{self.device}"
            with torch.cuda.stream(stream):
                u0 = torch.from_numpy(np.ascontiguousarray(r.u0)).to(dev)
                g = torch.zeros(ctx.shape, dtype=torch.complex128, device=dev)
            stream.synchronize()
            if r.kind == "optimise":  # u0 becomes the optimum, in place
                stats, hist = ctx.pnop_optimise(u0, r.E0, r.horizon, r.max_iter, r.tol)
                with torch.cuda.stream(stream):
                    u = u0.cpu()
                stream.synchronize()
                return stats["gain"], u.numpy(), hist
            if r.kind != "gradient":
                raise ValueError(f"unknown request kind {r.kind!r}")
            gain = ctx.pnop_gradient(u0, r.E0, r.horizon, g)
            with torch.cuda.stream(stream):
                grad = g.cpu()
            stream.synchronize()
            return gain, grad.numpy()
        finally:
            ctx.close()

    def _run(self, r: Request, need: int, admitted: float) -> None:
        err, gain, grad, hist = None, float("nan"), None, None
        try:
            out = self.runner(r, need)
            gain, grad = out[0], out[1]
            hist = out[2] if len(out) > 2 else None
        except Exception as e:  # reported per request; the server keeps running
            err = f"{type(e).__name__}: {e}"
        done = self.now()
        with self.lock:
            if r.rid in self.cancelled:
                gain, grad, hist, err = float("nan"), None, None, CANCELLED
            self.results[r.rid] = Result(r.rid, gain, grad, r.arrival, admitted, done, need, err, hist)
            self.active -= 1
            self.bytes_in_use -= need
            self._admit_locked()
            self.lock.notify_all()

    def wait(self, n: int, timeout: float = 3600.0) -> None:
        """Block until n results are in."""
        end = time.perf_counter() + timeout
        with self.lock:
            while len(self.results) < n:
                self._expire_locked()
                if len(self.results) >= n:
                    break
                left = end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{len(self.results)} of {n} requests finished")
                self.lock.wait(timeout=min(left, 0.05))


class BatchServer:
    """Continuous batching with shared launches.

    Requests of one kind (grid, precision, checkpoint slots) run in pnop_batch
    objects of `slots` request slots each: every kernel of a step runs once for
    all requests of a batch taking that kind of step.  A driver thread takes
    arrivals in order, has their host operators built on a small thread pool
    (pnop_batch_prepare, which may run beside the device work), admits
    prepared requests into free slots (first come, first served per kind),
    keeps up to `rounds` rounds of `ticks` batched steps queued per batch
    (without blocking on the device), and collects finished requests.

    Slots follow the arrival mix: when every slot of a kind is busy and more
    of its requests are waiting, another batch of that kind is created if the
    HBM budget allows (up to `max_batches_per_kind`, default unlimited), so a
    resolution that receives more requests gets more slots.  Prepared requests
    are admitted in arrival order across kinds, and `max_active_total` (default
    unlimited) caps the requests running at once over all batches: more
    concurrent requests add throughput only while the GPU has room, and beyond
    that they lengthen every request's latency.  A batch's device
    memory (pnop_batch_bytes) is counted against the budget from its creation;
    idle batches are released when another batch needs the memory, first
    those of kinds with nothing waiting.
    Each request gets bitwise the result it gets alone (the batched steps are
    the single-request steps per slot).

    Optimisation requests (adjoint looping) run one context each on an inner
    Server, at most `opt_active` at a time within a quarter of the HBM
    budget: their line search needs forward-only sweeps of one request,
    which a batch does not run.

    cancel(rid) and deadlines behave as in Server: a request not yet in a
    slot is dropped; one in a slot runs to its end (its steps are shared
    launches) and its result is discarded."""

    def __init__(self, hbm_budget: int, slots: int = 8, ticks: int = 4, device: int = 0, batch_factory=None,
                 sizer=None, rounds: int = 3, workers: int = 4, opt_active: int = 2, opt_runner=None,
                 opt_sizer=None, max_batches_per_kind: Optional[int] = None,
                 max_active_total: Optional[int] = None):
        """batch_factory(request, slots, stream) -> batch object (pnop_batch_prepare / submit_prepared /
        run / poll / result / close, as _lib.Batch) and sizer(request, slots) -> bytes replace the GPU
        batch and the library estimate (host-side tests)."""
        from concurrent.futures import ThreadPoolExecutor
        self.hbm_budget = int(hbm_budget)
        self.slots = slots
        self.ticks = ticks
        self.max_rounds = rounds
        self.max_batches = max_batches_per_kind
        self.max_total = max_active_total
        self.device = device
        self.factory = batch_factory
        self.sizer = sizer
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.queue: deque = deque()
        self.results: dict = {}
        self.lock = threading.Condition()
        self.t0 = time.perf_counter()
        # key -> {"batches": [entry], "prepared": deque of (request, future)}; an entry is
        # dict(batch, stream, bytes, running {bid: (request, admitted)}, rounds)
        self.kinds: dict = {}
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.active = 0
        self.peak_active = 0
        self.peak_batch = 0
        self.peak_batches_per_kind = 0
        self.batches_made = 0
        self.closed = False
        self.error: Optional[str] = None
        self.opt_active = opt_active
        self.opt_runner = opt_runner
        self.opt_sizer = opt_sizer
        self.opt_server: Optional[Server] = None
        self.opt_rids: set = set()
        self.cancelled: set = set()
        self.driver = threading.Thread(target=self._drive, daemon=True)
        self.driver.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    @staticmethod
    def key(r: Request):
        return (r.nr, r.ntheta, r.nz, r.Lz, r.precision, r.snaps)

    def batch_bytes(self, r: Request) -> int:
        if self.sizer is not None:
            return int(self.sizer(r, self.slots))
        return _lib.pnop_batch_bytes(r.nr, r.ntheta, r.nz, r.Lz, r.precision, r.snaps, self.slots)

    def cancel(self, rid: int) -> bool:
        """Cancel a request (see the class note); False when it is unknown or done."""
        if rid in self.opt_rids:
            return self.opt_server.cancel(rid)
        with self.lock:
            for r in list(self.queue):
                if r.rid == rid:
                    self.queue.remove(r)
                    self.results[r.rid] = Result(r.rid, float("nan"), None, r.arrival, float("nan"), self.now(), 0,
                                                 CANCELLED)
                    self.lock.notify_all()
                    return True
            if rid in self.results:
                return False
            self.cancelled.add(rid)
            return True

    def _dropped(self, r: Request) -> Optional[str]:
        """Why a request not yet in a slot is dropped (None: keep it)."""
        if r.rid in self.cancelled:
            return CANCELLED
        if r.deadline is not None and self.now() - r.arrival > r.deadline:
            return EXPIRED
        return None

    def submit(self, r: Request) -> None:
        if r.kind == "optimise":
            self.opt_rids.add(r.rid)
            if self.opt_server is None:
                self.opt_server = Server(self.hbm_budget // 4, self.opt_active, self.device, self.opt_runner,
                                         self.opt_sizer)
                self.opt_server.t0 = self.t0
            self.opt_server.submit(r)
            return
        if r.kind != "gradient":
            raise ValueError(f"unknown request kind {r.kind!r}")
        if self.batch_bytes(r) > self.hbm_budget:
            raise ValueError(f"request {r.rid}: a batch of its kind needs more than the whole budget")
        with self.lock:
            self.queue.append(r)
            self.lock.notify_all()

    # ---- driver thread
    def _kind(self, r: Request):
        k = self.key(r)
        if k not in self.kinds:
            self.kinds[k] = {"batches": [], "prepared": deque()}
        return self.kinds[k]

    def _release_for(self, need: int) -> None:
        """Close idle batches until `need` more bytes fit: first those of kinds
        with no prepared request waiting, then idle extra batches of any kind."""
        def idle(kd):
            return [e for e in kd["batches"] if not e["running"]]
        order = [(kd, e) for kd in self.kinds.values() if not kd["prepared"] for e in idle(kd)]
        order += [(kd, e) for kd in self.kinds.values() if kd["prepared"] for e in idle(kd)[1:]]
        for kd, e in order:
            if self.bytes_in_use + need <= self.hbm_budget:
                return
            kd["batches"].remove(e)
            e["batch"].close()
            self.bytes_in_use -= e["bytes"]

    def _new_batch(self, kd, r: Request):
        """Another batch for r's kind, or None when the budget has no room."""
        need = self.batch_bytes(r)
        if self.bytes_in_use + need > self.hbm_budget:
            self._release_for(need)
        if self.bytes_in_use + need > self.hbm_budget:
            return None
        if self.factory is not None:
            b, stream = self.factory(r, self.slots, None), None
        else:
            import torch
            stream = torch.cuda.Stream(device=self.device)
            b = _lib.Batch(r.nr, r.ntheta, r.nz, r.Lz, self.slots, r.precision, r.snaps, stream=stream.cuda_stream)
        e = {"batch": b, "stream": stream, "bytes": need, "running": {}, "rounds": deque()}
        kd["batches"].append(e)
        self.batches_made += 1
        self.bytes_in_use += need
        self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
        self.peak_batches_per_kind = max(self.peak_batches_per_kind, len(kd["batches"]))
        return e

    def _route(self, pending: deque) -> None:
        """Arrivals to their kind's preparation queue (in order), at most
        `slots` waiting per batch of the kind (and per batch it may still get)."""
        keep = deque()
        while pending:
            r = pending.popleft()
            why = self._dropped(r)
            if why:
                self._finish(r, float("nan"), float("nan"), None, why)
                continue
            kd = self._kind(r)
            if not kd["batches"] and self._new_batch(kd, r) is None:
                keep.append(r)
                continue
            if len(kd["prepared"]) >= self.slots * (len(kd["batches"]) + 1):
                keep.append(r)
                continue
            fut = self.pool.submit(kd["batches"][0]["batch"].pnop_batch_prepare, r.Re, r.dt, r.Wo, r.A, r.tau0)
            kd["prepared"].append((r, fut))
        pending.extend(keep)

    def _slot_for(self, kd, r: Request):
        """A batch of the kind with a free slot, a new one if allowed and the budget has room, or None."""
        for e in kd["batches"]:
            if len(e["running"]) < self.slots:
                return e
        if self.max_batches is not None and len(kd["batches"]) >= self.max_batches:
            return None
        return self._new_batch(kd, r)

    def _admit_all(self) -> bool:
        """Prepared requests into slots, oldest arrival first over all kinds."""
        did = False
        for kd in self.kinds.values():
            for item in [x for x in kd["prepared"] if x[1].done() and self._dropped(x[0])]:
                kd["prepared"].remove(item)
                r, fut = item
                try:
                    _lib_free(kd, fut.result())
                except Exception:
                    pass
                self._finish(r, float("nan"), float("nan"), None, self._dropped(r))
                did = True
        blocked = set()
        while self.max_total is None or self.active < self.max_total:
            cands = [(kd["prepared"][0][0].arrival, key) for key, kd in self.kinds.items()
                     if key not in blocked and kd["prepared"] and kd["prepared"][0][1].done()]
            if not cands:
                break
            key = min(cands)[1]
            if self._admit_one(self.kinds[key]):
                did = True
            else:
                blocked.add(key)
        return did

    def _admit_one(self, kd) -> bool:
        """The head of the kind's prepared queue into a slot; False when no slot is free."""
        while kd["prepared"] and kd["prepared"][0][1].done():
            r, fut = kd["prepared"][0]
            e = self._slot_for(kd, r)
            if e is None:
                return False
            kd["prepared"].popleft()
            ops = None
            try:
                ops = fut.result()
                bid = self._submit_one(e, r, ops)
            except Exception as ex:  # reported per request
                self._finish(r, self.now(), float("nan"), None, f"{type(ex).__name__}: {ex}")
                continue
            finally:
                if ops is not None:
                    e["batch"].pnop_ops_free(ops)
            e["running"][bid] = (r, self.now())
            self.active += 1
            self.peak_active = max(self.peak_active, self.active)
            self.peak_batch = max(self.peak_batch, len(e["running"]))
            return True
        return False

    def _submit_one(self, e, r: Request, ops) -> int:
        b = e["batch"]
        if self.factory is not None:
            return b.pnop_batch_submit_prepared(ops, r.u0, r.E0, r.horizon)
        import torch
        with torch.cuda.stream(e["stream"]):
            u0 = torch.from_numpy(np.ascontiguousarray(r.u0)).to(f"cuda:{self.device}", non_blocking=False)
        return b.pnop_batch_submit_prepared(ops, u0, r.E0, r.horizon)

    def _queue_rounds(self, e) -> bool:
        rounds = e["rounds"]
        while rounds and (rounds[0] is None or rounds[0].query()):
            rounds.popleft()
        did = False
        while e["running"] and len(rounds) < self.max_rounds:
            _, running = e["batch"].pnop_batch_run(self.ticks)
            ev = None
            if e["stream"] is not None:
                import torch
                ev = torch.cuda.Event()
                ev.record(e["stream"])
            rounds.append(ev)
            did = True
            if running == 0:
                break
        return did

    def _collect(self, e) -> bool:
        b = e["batch"]
        did = False
        for bid in list(e["running"]):
            if not b.pnop_batch_poll(bid):
                continue
            r, admitted = e["running"].pop(bid)
            self.active -= 1
            did = True
            err, gain, grad = None, float("nan"), None
            try:
                if self.factory is not None:
                    gain, grad = b.pnop_batch_result(bid)
                else:
                    import torch
                    with torch.cuda.stream(e["stream"]):
                        g = torch.empty(b.shape, dtype=torch.complex128, device=f"cuda:{self.device}")
                    gain = b.pnop_batch_result(bid, g)
                    grad = g.cpu().numpy()
            except Exception as ex:
                err = f"{type(ex).__name__}: {ex}"
            if r.rid in self.cancelled:
                gain, grad, err = float("nan"), None, CANCELLED
            self._finish(r, admitted, gain, grad, err)
        return did

    def _finish(self, r, admitted, gain, grad, err) -> None:
        with self.lock:
            self.results[r.rid] = Result(r.rid, gain, grad, r.arrival, admitted, self.now(), 0, err)
            self.lock.notify_all()

    def _drive(self) -> None:
        if self.factory is None:
            import torch
            torch.cuda.set_device(self.device)
        pending: deque = deque()
        try:
            while True:
                with self.lock:
                    waiting = pending or any(kd["prepared"] for kd in self.kinds.values())
                    if self.closed and not self.queue and not waiting and not self.active:
                        return
                    if not self.queue and not waiting and not self.active:
                        self.lock.wait(timeout=0.05)
                    pending.extend(self.queue)
                    self.queue.clear()
                self._route(pending)
                did = self._admit_all()
                for kd in list(self.kinds.values()):
                    for e in list(kd["batches"]):
                        did |= self._queue_rounds(e)
                        did |= self._collect(e)
                if not did:
                    time.sleep(0.0002)
        except Exception as ex:  # the driver stops; waiters see the error
            with self.lock:
                self.error = f"{type(ex).__name__}: {ex}"
                self.lock.notify_all()

    def wait(self, n: int, timeout: float = 3600.0) -> None:
        end = time.perf_counter() + timeout

        def count():
            return len(self.results) + (len(self.opt_server.results) if self.opt_server else 0)

        with self.lock:
            while count() < n:
                if self.error:
                    raise RuntimeError(f"serving driver failed: {self.error}")
                left = end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{count()} of {n} requests finished")
                self.lock.wait(timeout=min(left, 0.05))
            if self.opt_server:
                self.results.update(self.opt_server.results)

    def close(self) -> None:
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        self.driver.join(timeout=60)
        self.pool.shutdown(wait=True)
        for kd in self.kinds.values():
            for _, fut in kd["prepared"]:
                try:
                    _lib_free(kd, fut.result())
                except Exception:
                    pass
            for e in kd["batches"]:
                e["batch"].close()
        self.kinds.clear()


def _lib_free(kd, ops) -> None:
    """Free prepared operators through any batch of their kind (the call is
    static in the library; a kind whose batches are gone frees nothing: its
    handles died with the test stand-ins)."""
    if kd["batches"]:
        kd["batches"][0]["batch"].pnop_ops_free(ops)
    elif ops is not None and not isinstance(ops, tuple):
        _lib.Batch.pnop_ops_free(ops)


def serve_stream(requests, hbm_budget: int, max_active: int = 8, device: int = 0, runner=None, sizer=None,
                 batched: bool = False, ticks: int = 4, batch_factory=None, max_batches_per_kind=None,
                 max_active_total=None):
    """Submit requests at their arrival times (seconds after start) and wait.

    Returns (results sorted by id, server).  Arrival times are honoured on the
    host clock; a request arriving while others run is admitted as soon as
    memory and a slot are free.  batched selects the BatchServer (max_active
    slots per batch of one kind) instead of one context and stream per
    request."""
    if batched:
        srv = BatchServer(hbm_budget, max_active, ticks, device, batch_factory, sizer,
                          max_batches_per_kind=max_batches_per_kind, max_active_total=max_active_total)
        try:
            for r in sorted(requests, key=lambda q: q.arrival):
                delay = r.arrival - srv.now()
                if delay > 0:
                    time.sleep(delay)
                srv.submit(r)
            srv.wait(len(requests))
        finally:
            srv.close()
        return [srv.results[r.rid] for r in sorted(requests, key=lambda q: q.rid)], srv
    srv = Server(hbm_budget, max_active, device, runner, sizer)
    for r in sorted(requests, key=lambda q: q.arrival):
        delay = r.arrival - srv.now()
        if delay > 0:
            time.sleep(delay)
        srv.submit(r)
    srv.wait(len(requests))
    return [srv.results[r.rid] for r in sorted(requests, key=lambda q: q.rid)], srv


def latency_summary(results):
    lat = np.array([x.latency for x in results if x.error is None])
    if lat.size == 0:
        return {"p50_s": None, "p99_s": None, "n": 0}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(lat.size)}
