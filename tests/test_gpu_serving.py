"""Serving on the GPU: requests of mixed resolution, precision and physics run
concurrently (admitted while others are on the device) and each result equals
the result of the same request run alone; one FP64 request is checked against
the oracle."""
import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib, serving
    return _lib, serving


def _requests(L, serving):
    specs = [  # (nr, ntheta, nz, Lz, Re, Wo, A, E0, nsteps, precision)
        (16, 8, 16, 10.0, 1800.0, 6.0, 0.8, 1e-4, 12, L.PNOP_FP64),
        (12, 16, 12, 7.0, 2500.0, 12.0, 1.2, 1e-5, 9, L.PNOP_MIXED),
        (16, 8, 16, 10.0, 1500.0, 4.0, 0.5, 1e-6, 15, L.PNOP_MIXED),
        (12, 16, 12, 7.0, 3000.0, 18.0, 1.5, 1e-7, 7, L.PNOP_FP64),
        (16, 8, 16, 10.0, 2200.0, 8.0, 1.0, 1e-5, 10, L.PNOP_MIXED),
    ]
    reqs = []
    for i, (nr, nth, nz, Lz, Re, Wo, A, E0, n, prec) in enumerate(specs):
        M, K = nth // 2 - 1, nz // 2 - 1
        r = po.radial_grid(nr)
        u0 = synth.random_field(r, M, K, Lz, seed=40 + i)
        reqs.append(serving.Request(rid=i, nr=nr, ntheta=nth, nz=nz, Lz=Lz, Re=Re, Wo=Wo, A=A, tau0=0.3 * i, E0=E0,
                                    horizon=n * 0.005, dt=0.005, u0=u0, precision=prec, snaps=3,
                                    arrival=0.004 * i))
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix(mods):
    L, serving = mods
    reqs = _requests(L, serving)
    mix, srv = serving.serve_stream(reqs, hbm_budget=8 << 30, max_active=5)
    assert all(r.error is None for r in mix), [r.error for r in mix]
    assert srv.peak_active >= 2  # the requests overlapped
    for r in reqs:
        alone, _ = serving.serve_stream([r], hbm_budget=8 << 30, max_active=1)
        a, m = alone[0], mix[r.rid]
        assert a.gain == m.gain
        assert np.array_equal(a.grad, m.grad)


def test_fp64_request_matches_the_oracle(mods):
    L, serving = mods
    r = _requests(L, serving)[0]
    res, _ = serving.serve_stream([r], hbm_budget=8 << 30)
    o = po.Oracle(po.Params(nr=r.nr, M=r.ntheta // 2 - 1, K=r.nz // 2 - 1, Lz=r.Lz, Re=r.Re, dt=r.dt, Wo=r.Wo, A=r.A))
    u0 = o.scale_to(r.u0, r.E0)
    n = int(round(r.horizon / r.dt))
    ET, g = o.gradient(u0, r.tau0, n)
    assert abs(res[0].gain / (ET / r.E0) - 1) < 1e-10
    assert np.abs(res[0].grad - g).max() <= 1e-10 * np.abs(g).max()


def test_admission_budget_serialises_when_memory_is_short(mods):
    L, serving = mods
    reqs = _requests(L, serving)[:3]
    need = max(L.pnop_context_bytes(r.nr, r.ntheta, r.nz, r.Lz, r.precision, r.snaps) for r in reqs)
    res, srv = serving.serve_stream(reqs, hbm_budget=need, max_active=8)
    assert all(r.error is None for r in res)
    assert srv.peak_active == 1


def test_batched_server_gives_each_request_its_alone_result(mods):
    L, serving = mods
    reqs = _requests(L, serving)
    for r in reqs:  # all at once, so that requests of one kind certainly share a batch
        r.arrival = 0.0
    mix, srv = serving.serve_stream(reqs, hbm_budget=8 << 30, max_active=4, batched=True, ticks=3)
    assert all(r.error is None for r in mix), [r.error for r in mix]
    assert srv.peak_batch >= 2  # requests of one kind shared launches
    for r in reqs:
        alone, _ = serving.serve_stream([r], hbm_budget=8 << 30, max_active=1)
        a, m = alone[0], mix[r.rid]
        assert a.gain == m.gain
        assert np.array_equal(a.grad, m.grad)


def test_optimisation_request_served_beside_gradients_matches_alone(mods):
    L, serving = mods
    import torch
    reqs = _requests(L, serving)[:3]
    for r in reqs:
        r.arrival = 0.0
    opt = reqs[1]
    opt.kind, opt.max_iter = "optimise", 2
    mix, srv = serving.serve_stream(reqs, hbm_budget=8 << 30, max_active=4, batched=True, ticks=3)
    assert all(r.error is None for r in mix), [r.error for r in mix]
    m = mix[opt.rid]
    assert m.history is not None and len(m.history) >= 2 and m.gain == m.history[-1]
    ctx = L.Context(opt.nr, opt.ntheta, opt.nz, opt.Lz, opt.Re, opt.dt, opt.Wo, opt.A, opt.tau0, opt.precision,
                    opt.snaps)
    u = torch.from_numpy(np.ascontiguousarray(opt.u0)).to("cuda")
    stats, hist = ctx.pnop_optimise(u, opt.E0, opt.horizon, opt.max_iter, opt.tol)
    ctx.close()
    assert m.gain == stats["gain"] and list(m.history) == list(hist)
    assert np.array_equal(m.grad, u.cpu().numpy())
    for r in (reqs[0], reqs[2]):
        alone, _ = serving.serve_stream([r], hbm_budget=8 << 30, max_active=1)
        assert alone[0].gain == mix[r.rid].gain and np.array_equal(alone[0].grad, mix[r.rid].grad)
