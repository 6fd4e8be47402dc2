"""Two-level checkpointing (Section 2.5, Eq. 2.21) with the second level in
pinned host memory: the gradient is bitwise the one of the single-level
schedule, and the sweep runs the schedule the host-side cost model chose."""
import math

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


def grads(L, nr, nth, nz, Lz, N, snaps, host_max, ratio, precision=0, seed=0):
    import torch
    out = []
    for hm in (0, host_max):
        ctx = L.Context(nr, nth, nz, Lz, 2000.0, 0.01, 8.0, 1.0, 0.0, precision, snaps)
        if hm:
            ctx.pnop_set_host_tier(hm, ratio)
        r = np.array(ctx.pnop_grid_points())
        u0 = torch.from_numpy(synth.random_field(r, nth // 2 - 1, nz // 2 - 1, Lz, seed=seed)).to("cuda")
        g = torch.zeros_like(u0)
        gain = ctx.pnop_gradient(u0, 1e-4, N * 0.01, g)
        out.append((gain, g.cpu().numpy(), ctx.pnop_gradient_stats(), ctx.pnop_host_tier_stats()))
        ctx.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_host_tier_gradient_is_bitwise_single_level(L, precision):
    N, s, H = 30, 2, 10
    (g0, d0, st0, _), (g1, d1, st1, ht) = grads(L, 12, 8, 12, 10.0, N, s, H, 0.0, precision)
    assert g0 == g1 and np.array_equal(d0, d1)
    nf, adv = L.pnop_two_level_counts(N, s, H, 0.0)
    assert nf > 0 and ht["host_checkpoints"] == nf
    assert ht["host_stores"] == nf and ht["host_loads"] == nf
    assert st1[0] == adv < st0[0]           # fewer forward steps than the single level
    assert st1[1] == st0[1] == N            # one adjoint step per step


@pytest.mark.parametrize("precision", [0, 1])
def test_host_tier_gradient_matches_the_oracle(L, precision):
    """The two-level sweep against the oracle's store-all gradient (not only
    against the single-level GPU sweep): FP64 to 1e-10, mixed precision within
    the mixed-precision budget (gain 1e-5, cosine 0.99999)."""
    N, s, H, E0 = 30, 2, 10, 1e-4
    (gain, g, st, ht) = grads(L, 12, 8, 12, 10.0, N, s, H, 0.0, precision)[1]
    assert ht["host_checkpoints"] > 0
    o = po.Oracle(po.Params(nr=12, M=3, K=5, Lz=10.0, Re=2000.0, dt=0.01, Wo=8.0, A=1.0))
    u0 = o.scale_to(synth.random_field(o.r, 3, 5, 10.0, seed=0), E0)
    ET, gref = o.gradient(u0, 0.0, N)
    if precision == 0:
        assert abs(gain / (ET / E0) - 1) < 1e-10
        assert np.abs(g - gref).max() <= 1e-10 * np.abs(gref).max()
    else:
        cos = o.inner(g, gref) / math.sqrt(o.inner(g, g) * o.inner(gref, gref))
        assert abs(gain / (ET / E0) - 1) <= 1e-5
        assert cos >= 0.99999


def test_host_tier_full_size_store_all_on_host(L):
    N = 12
    (g0, d0, st0, _), (g1, d1, st1, ht) = grads(L, 64, 64, 256, 100.0, N, 2, N - 1, 0.0, precision=1)
    assert g0 == g1 and np.array_equal(d0, d1)
    assert st1[0] == N                     # every state computed once
    assert ht["host_checkpoints"] >= N - 2


def test_host_tier_measures_its_io_ratio(L):
    ctx = L.Context(16, 16, 32, 10.0, 2000.0, 0.01, 8.0, 1.0, 0.0, 1, 2)
    ctx.pnop_set_host_tier(8, -1.0)
    r = ctx.pnop_host_tier_stats()["io_ratio"]
    assert math.isfinite(r) and r > 0
    ctx.close()
