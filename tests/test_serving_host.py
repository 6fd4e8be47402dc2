"""Host-side behaviour of the continuous-batching server (no GPU): admission
by HBM budget and slot count, late arrivals joining running work, errors
reported per request."""
import threading
import time

import numpy as np
import pytest

from paper_2509_10103_gb300 import serving


def _req(i, arrival=0.0, size=1):
    return serving.Request(rid=i, nr=size, ntheta=4, nz=4, Lz=1.0, Re=1.0, Wo=1.0, A=0.0, tau0=0.0, E0=1.0,
                           horizon=1.0, dt=1.0, u0=np.zeros(1), arrival=arrival)


class FakeGPU:
    def __init__(self, dur=0.05):
        self.dur = dur
        self.lock = threading.Lock()
        self.live = 0
        self.peak = 0
        self.start = {}

    def __call__(self, r, need):
        with self.lock:
            self.live += 1
            self.peak = max(self.peak, self.live)
            self.start[r.rid] = time.perf_counter()
        time.sleep(self.dur)
        with self.lock:
            self.live -= 1
        if r.rid == 13:
            raise RuntimeError("planted failure")
        return float(r.rid), np.full(3, r.rid)


def test_admission_respects_budget_and_slots():
    gpu = FakeGPU()
    reqs = [_req(i, size=1 + i % 3) for i in range(12)]
    res, srv = serving.serve_stream(reqs, hbm_budget=4, max_active=3, runner=gpu, sizer=lambda r: r.nr)
    assert len(res) == 12 and all(x.error is None for x in res)
    assert srv.peak_bytes <= 4 and srv.peak_active <= 3 and gpu.peak <= 3
    assert srv.bytes_in_use == 0 and srv.active == 0
    assert [x.gain for x in res] == [float(i) for i in range(12)]


def test_late_arrival_joins_running_work():
    gpu = FakeGPU(dur=0.3)
    reqs = [_req(0, 0.0), _req(1, 0.1)]
    res, srv = serving.serve_stream(reqs, hbm_budget=10, max_active=4, runner=gpu, sizer=lambda r: 1)
    # the second request starts while the first is still on the "device"
    assert gpu.start[1] - gpu.start[0] < 0.25
    assert gpu.peak == 2
    assert res[1].admitted - res[1].arrival < 0.05


def test_request_larger_than_budget_is_refused_and_errors_are_per_request():
    with pytest.raises(ValueError):
        serving.Server(hbm_budget=1, runner=FakeGPU(), sizer=lambda r: 5).submit(_req(0))
    gpu = FakeGPU(dur=0.01)
    res, _ = serving.serve_stream([_req(12), _req(13), _req(14)], hbm_budget=3, max_active=3, runner=gpu,
                                  sizer=lambda r: 1)
    assert res[1].error and "planted" in res[1].error
    assert res[0].error is None and res[2].error is None


def test_latency_summary():
    rs = [serving.Result(i, 1.0, None, 0.0, 0.0, float(i + 1), 0) for i in range(100)]
    s = serving.latency_summary(rs)
    assert abs(s["p50_s"] - 50.5) < 1e-9 and s["p99_s"] > 99.0 and s["n"] == 100


class FakeBatch:
    """Stands in for a pnop_batch: a request finishes after as many ticks as
    its horizon has steps; each tick covers every unfinished request."""
    made = []

    def __init__(self, r, slots, stream):
        self.slots = slots
        self.left = {}
        self.gain = {}
        self.next = 0
        self.max_live = 0
        self.closed = False
        FakeBatch.made.append(self)

    def pnop_batch_prepare(self, Re, dt, Wo, A, tau0):
        if Re < 0:
            raise RuntimeError("planted failure")
        return (Re, dt)

    @staticmethod
    def pnop_ops_free(ops):
        pass

    def pnop_batch_submit_prepared(self, ops, u0, E0, horizon):
        assert len(self.left) < self.slots
        Re, dt = ops
        bid = self.next
        self.next += 1
        self.left[bid] = int(round(horizon / dt))
        self.gain[bid] = Re
        return bid

    def pnop_batch_run(self, ticks):
        for _ in range(ticks):
            live = [b for b, n in self.left.items() if n > 0]
            self.max_live = max(self.max_live, len(live))
            for b in live:
                self.left[b] -= 1
        return ticks, sum(1 for n in self.left.values() if n > 0)

    def pnop_batch_poll(self, bid):
        return self.left[bid] == 0

    def pnop_batch_result(self, bid):
        del self.left[bid]
        return self.gain.pop(bid), np.full(3, bid)

    def close(self):
        self.closed = True


def _breq(i, kind, steps, arrival=0.0, Re=None):
    r = _req(i, arrival, size=kind)
    r.horizon = float(steps)
    r.Re = float(i) if Re is None else Re
    return r


def test_batch_server_shares_steps_and_respects_slots():
    FakeBatch.made.clear()
    reqs = [_breq(i, 1 + i % 2, 3 + i % 5) for i in range(14)]
    res, srv = serving.serve_stream(reqs, hbm_budget=10, max_active=3, batched=True, ticks=1,
                                    batch_factory=FakeBatch, sizer=lambda r, slots: 1, max_batches_per_kind=1)
    assert all(x.error is None for x in res), [x.error for x in res]
    assert [x.gain for x in res] == [float(i) for i in range(14)]
    assert len(FakeBatch.made) == 2  # one batch per kind of request
    assert all(b.max_live <= 3 for b in FakeBatch.made)  # slot limit
    assert max(b.max_live for b in FakeBatch.made) >= 2  # requests shared ticks
    assert srv.peak_batch <= 3 and srv.active == 0


def test_batch_server_slots_follow_the_arrival_mix():
    """Nine requests of one kind and one of another arrive at once: the busy
    kind gets further batches (its waiting requests take new slots instead of
    queueing), the other keeps one, and the budget bounds the total."""
    FakeBatch.made.clear()
    reqs = [_breq(i, 1, 16) for i in range(9)] + [_breq(9, 2, 16)]
    res, srv = serving.serve_stream(reqs, hbm_budget=4, max_active=3, batched=True, ticks=1,
                                    batch_factory=SlowerBatch, sizer=lambda r, slots: 1)
    assert all(x.error is None for x in res), [x.error for x in res]
    assert [x.gain for x in res] == [float(i) for i in range(10)]
    assert srv.peak_batches_per_kind == 3          # 9 requests / 3 slots (each holds its slot ~0.8 s)
    assert srv.peak_bytes <= 4 and len(FakeBatch.made) == 4
    assert all(b.max_live <= 3 for b in FakeBatch.made)


def test_batch_server_caps_concurrency_and_admits_in_arrival_order():
    """With max_active_total, at most that many requests run over all batches,
    and waiting requests enter slots oldest first whatever their kind."""
    FakeBatch.made.clear()
    reqs = [_breq(i, 1 + (i % 2), 6, arrival=0.001 * i) for i in range(8)]
    res, srv = serving.serve_stream(reqs, hbm_budget=8, max_active=4, batched=True, ticks=1,
                                    batch_factory=SlowBatch, sizer=lambda r, slots: 1, max_active_total=2)
    assert all(x.error is None for x in res), [x.error for x in res]
    assert srv.peak_active == 2
    admitted = sorted(range(8), key=lambda i: res[i].admitted)
    assert admitted == list(range(8))


def test_batch_server_budget_releases_idle_batches_and_reports_errors():
    FakeBatch.made.clear()
    reqs = [_breq(0, 1, 4), _breq(1, 2, 4, arrival=0.05), _breq(2, 1, 2, arrival=0.1, Re=-1.0)]
    # room for one batch at a time: kind 2 waits for kind 1's batch to go idle
    res, srv = serving.serve_stream(reqs, hbm_budget=1, max_active=2, batched=True, ticks=1,
                                    batch_factory=FakeBatch, sizer=lambda r, slots: 1)
    assert res[0].error is None and res[1].error is None
    assert res[2].error is not None and "planted" in res[2].error
    assert srv.peak_bytes <= 1
    assert len(FakeBatch.made) == 3 and FakeBatch.made[0].closed


def test_batch_server_runs_optimisation_requests_on_contexts():
    FakeBatch.made.clear()
    seen = []

    def opt_runner(r, need):
        seen.append(r.rid)
        time.sleep(0.02)
        return 100.0 + r.rid, np.full(3, -r.rid), [1.0, 50.0, 100.0 + r.rid]

    srv = serving.BatchServer(hbm_budget=8, slots=2, ticks=1, batch_factory=FakeBatch,
                              sizer=lambda r, slots: 1, opt_runner=opt_runner, opt_sizer=lambda r: 1)
    reqs = [_breq(i, 1, 3) for i in range(6)]
    for r in reqs[::2]:
        r.kind = "optimise"
    try:
        for r in reqs:
            srv.submit(r)
        srv.wait(len(reqs))
    finally:
        srv.close()
    res = srv.results
    assert sorted(seen) == [0, 2, 4]
    for i in range(6):
        assert res[i].error is None
        if i % 2 == 0:
            assert res[i].gain == 100.0 + i and res[i].history[-1] == res[i].gain
        else:
            assert res[i].gain == float(i) and res[i].history is None
    with pytest.raises(ValueError):
        bad = _breq(9, 1, 3)
        bad.kind = "bogus"
        srv.submit(bad)


def test_context_server_cancels_and_expires_requests():
    gpu = FakeGPU(dur=0.2)
    srv = serving.Server(hbm_budget=1, max_active=1, runner=gpu, sizer=lambda r: 1)
    reqs = [_req(0), _req(1), _req(2), _req(3)]
    reqs[3].deadline = 0.05            # waits behind request 0 and 2 for longer than 50 ms
    for r in reqs:
        srv.submit(r)
    assert srv.cancel(1)               # queued: dropped at once
    assert srv.cancel(0)               # running: finishes, result discarded
    srv.wait(4)
    res = srv.results
    assert res[0].error == serving.CANCELLED and res[0].grad is None
    assert res[1].error == serving.CANCELLED and res[1].rid not in gpu.start
    assert res[2].error is None and res[2].gain == 2.0
    assert res[3].error == serving.EXPIRED and 3 not in gpu.start
    assert not srv.cancel(2)           # already done


class SlowBatch(FakeBatch):
    """FakeBatch whose ticks take real time, so that requests wait for slots."""

    def pnop_batch_run(self, ticks):
        time.sleep(0.01 * ticks)
        return super().pnop_batch_run(ticks)


class SlowerBatch(FakeBatch):
    """Ticks of 50 ms: every request of a burst is prepared long before the
    first one could free its slot, even on a loaded host."""

    def pnop_batch_run(self, ticks):
        time.sleep(0.05 * ticks)
        return super().pnop_batch_run(ticks)


def test_batch_server_cancels_and_expires_requests():
    FakeBatch.made.clear()
    srv = serving.BatchServer(hbm_budget=8, slots=1, ticks=1, batch_factory=SlowBatch, sizer=lambda r, slots: 1,
                              max_batches_per_kind=1)
    reqs = [_breq(0, 1, 20), _breq(1, 1, 3), _breq(2, 1, 3), _breq(3, 1, 3)]
    reqs[3].deadline = 0.05            # one slot, busy with request 0 for ~0.2 s
    try:
        for r in reqs:
            srv.submit(r)
        time.sleep(0.02)
        assert srv.cancel(0)           # in its slot: runs to the end, result discarded
        assert srv.cancel(1)           # waiting for the slot: dropped
        srv.wait(4)
    finally:
        srv.close()
    res = srv.results
    assert res[0].error == serving.CANCELLED and res[0].grad is None
    assert res[1].error == serving.CANCELLED
    assert res[2].error is None and res[2].gain == 2.0
    assert res[3].error == serving.EXPIRED
