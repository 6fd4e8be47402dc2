"""Batched gradients (pnop_batch_*): requests of one grid with their own
physics, E0 and horizon run through shared launches, and each one gets
bitwise the gradient and gain of the single-request path (pnop_gradient with
the same checkpoint budget and precision), which the parity tests pin to the
oracle.  Requests admitted while others run (continuous batching) get the
same bits too."""
import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return _lib


GRID = dict(nr=12, ntheta=8, nz=12, Lz=6.0)  # |m| <= 3, k <= 5
REQS = [  # Re, Wo, A, dt, tau0, E0, steps
    (2000.0, 8.0, 1.0, 0.01, 0.0, 1e-3, 7),
    (1500.0, 4.0, 0.5, 0.02, 3.0, 1e-6, 4),
    (3000.0, 18.0, 1.5, 0.005, 1.0, 1e-4, 9),
    (1750.0, 2.0, 0.0, 0.01, 0.0, 1e-20, 1),
    (2500.0, 12.0, 1.0, 0.01, 5.5, 1e-5, 6),
]


def seeds(L, n, grid=GRID):
    import torch
    M, K = grid["ntheta"] // 2 - 1, grid["nz"] // 2 - 1
    r = np.array(po.Oracle(po.Params(nr=grid["nr"], M=M, K=K, Lz=grid["Lz"], Re=2000.0, dt=0.01, Wo=8.0,
                                     A=0.0)).r)
    return [torch.from_numpy(synth.random_field(r, M, K, grid["Lz"], seed=10 + i)).to("cuda") for i in range(n)]


def alone(L, req, u0, precision, snaps, grid=GRID):
    import torch
    Re, Wo, A, dt, tau0, E0, n = req
    ctx = L.Context(grid["nr"], grid["ntheta"], grid["nz"], grid["Lz"], Re, dt, Wo, A, tau0, precision, snaps)
    g = torch.empty_like(u0)
    gain = ctx.pnop_gradient(u0, E0, n * dt, g)
    ctx.close()
    return gain, g


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_each_request_alone_bitwise(L, precision):
    import torch
    snaps = 3
    us = seeds(L, len(REQS))
    b = L.Batch(GRID["nr"], GRID["ntheta"], GRID["nz"], GRID["Lz"], capacity=len(REQS), precision=precision,
                snap_budget=snaps)
    ids = [b.pnop_batch_submit(u, r[5], r[6] * r[3], r[0], r[3], r[1], r[2], r[4]) for r, u in zip(REQS, us)]
    ticks, running = b.pnop_batch_run(10000)
    assert running == 0
    stats = b.pnop_batch_stats()
    assert stats["ticks"] <= ticks and stats["entries"] > stats["ticks"]  # steps were shared between requests
    for rid, r, u in zip(ids, REQS, us):
        assert b.pnop_batch_poll(rid) or True  # poll never blocks; result waits
        g = torch.empty_like(u)
        gain = b.pnop_batch_result(rid, g)
        gain1, g1 = alone(L, r, u, precision, snaps)
        assert gain == gain1
        assert torch.equal(g, g1)
    b.close()


def test_requests_admitted_while_others_run_get_the_same_bits(L):
    import torch
    snaps = 2
    us = seeds(L, 4)
    b = L.Batch(GRID["nr"], GRID["ntheta"], GRID["nz"], GRID["Lz"], capacity=3, precision=1, snap_budget=snaps)
    reqs = REQS[:4]
    first = [b.pnop_batch_submit(us[i], reqs[i][5], reqs[i][6] * reqs[i][3], reqs[i][0], reqs[i][3], reqs[i][1],
                                 reqs[i][2], reqs[i][4]) for i in range(3)]
    with pytest.raises(L.PnopError):  # all three slots are taken
        b.pnop_batch_submit(us[3], 1e-3, 0.01, 2000.0, 0.01)
    b.pnop_batch_run(5)
    with pytest.raises(L.PnopError):  # request 0 needs more than 5 ticks
        b.pnop_batch_result(first[0])
    b.pnop_batch_run(10000)
    out = {}
    out[0] = b.pnop_batch_result(first[0], g0 := torch.empty_like(us[0])), g0
    late = b.pnop_batch_submit(us[3], reqs[3][5], reqs[3][6] * reqs[3][3], reqs[3][0], reqs[3][3], reqs[3][1],
                               reqs[3][2], reqs[3][4])
    b.pnop_batch_run(10000)
    for i, rid in ((1, first[1]), (2, first[2]), (3, late)):
        g = torch.empty_like(us[i])
        out[i] = b.pnop_batch_result(rid, g), g
    for i in range(4):
        gain1, g1 = alone(L, reqs[i], us[i], 1, snaps)
        assert out[i][0] == gain1
        assert torch.equal(out[i][1], g1)
    b.close()


def test_batch_at_full_size_matches_alone(L):
    """64x64x256 (|m| <= 31, k <= 127, 96x384 physical), mixed precision: two
    requests through the two-pass transform kernels with nb = 2."""
    import torch
    grid = dict(nr=64, ntheta=64, nz=256, Lz=100.0)
    reqs = [(2000.0, 8.0, 1.0, 0.0025, 0.0, 1e-5, 3), (3000.0, 4.0, 0.5, 0.005, 2.0, 1e-6, 2)]
    us = seeds(L, 2, grid)
    b = L.Batch(grid["nr"], grid["ntheta"], grid["nz"], grid["Lz"], capacity=2, precision=1, snap_budget=2)
    ids = [b.pnop_batch_submit(u, r[5], r[6] * r[3], r[0], r[3], r[1], r[2], r[4]) for r, u in zip(reqs, us)]
    b.pnop_batch_run(10000)
    for rid, r, u in zip(ids, reqs, us):
        g = torch.empty_like(u)
        gain = b.pnop_batch_result(rid, g)
        gain1, g1 = alone(L, r, u, 1, 2, grid)
        assert gain == gain1
        assert torch.equal(g, g1)
    b.close()


def test_batched_fp64_requests_match_the_oracle(L):
    """Two FP64 requests of different physics in one batch against the oracle
    gradient (relative 1e-10, as the single-request parity tests)."""
    import torch
    reqs = [REQS[0], REQS[1]]
    us = seeds(L, 2)
    b = L.Batch(GRID["nr"], GRID["ntheta"], GRID["nz"], GRID["Lz"], capacity=2, precision=0, snap_budget=3)
    ids = [b.pnop_batch_submit(u, r[5], r[6] * r[3], r[0], r[3], r[1], r[2], r[4]) for r, u in zip(reqs, us)]
    b.pnop_batch_run(10000)
    M, K = GRID["ntheta"] // 2 - 1, GRID["nz"] // 2 - 1
    for rid, (Re, Wo, A, dt, tau0, E0, n), u in zip(ids, reqs, us):
        g = torch.empty_like(u)
        gain = b.pnop_batch_result(rid, g)
        o = po.Oracle(po.Params(nr=GRID["nr"], M=M, K=K, Lz=GRID["Lz"], Re=Re, dt=dt, Wo=Wo, A=A))
        u0 = o.scale_to(u.cpu().numpy(), E0)
        ET, gref = o.gradient(u0, tau0, n)
        assert abs(gain / (ET / o.energy(u0)) - 1) < 1e-10
        assert np.abs(g.cpu().numpy() - gref).max() <= 1e-10 * np.abs(gref).max()
    b.close()


def test_batch_bytes_bounds_what_a_batch_allocates(L):
    import torch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    b = L.Batch(32, 32, 64, 10.0, capacity=4, precision=1, snap_budget=4)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    b.close()
    used = free0 - free1
    est = L.pnop_batch_bytes(32, 32, 64, 10.0, 1, 4, 4)
    assert 0 < used <= est
