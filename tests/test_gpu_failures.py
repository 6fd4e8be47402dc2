"""Failure detection without any GPU fault: a host-side deadline on device
waits returns PNOP_ERR_TIMEOUT and leaves the context usable; a non-finite
input is reported as PNOP_ERR_NONFINITE; an HBM budget too small for the
checkpoint pool is reported as PNOP_ERR_OOM."""
import math

import numpy as np
import pytest

from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return torch, _lib


def _ctx(L, **kw):
    a = dict(nr=32, ntheta=16, nz=32, Lz=10.0, Re=2000.0, dt=0.01)
    return L.Context(a["nr"], a["ntheta"], a["nz"], a["Lz"], a["Re"], a["dt"], 8.0, 1.0, 0.0, kw.get("precision", 0),
                     kw.get("snaps", 4), hbm_budget=kw.get("hbm", 0))


def test_timeout_then_recover(env):
    torch, L = env
    ctx = _ctx(L)
    r = np.array(ctx.pnop_grid_points())
    u0 = torch.from_numpy(synth.random_field(r, ctx.M, ctx.K, 10.0, seed=1)).to("cuda")
    g = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    ref = ctx.pnop_gradient(u0, 1e-4, 0.5, g)
    ctx.pnop_set_timeout(1e-6)  # far shorter than a 50-step gradient
    with pytest.raises(L.PnopError) as e:
        ctx.pnop_gradient(u0, 1e-4, 0.5, g)
    assert e.value.code == -5
    ctx.pnop_sync()             # the queued work finishes; nothing was aborted
    ctx.pnop_set_timeout(0.0)
    again = ctx.pnop_gradient(u0, 1e-4, 0.5, g)
    assert again == ref
    ctx.close()


def test_nonfinite_input_is_reported(env):
    torch, L = env
    ctx = _ctx(L)
    u = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    u[2, 5, ctx.M + 1, 3] = complex(float("nan"), 0.0)
    g = torch.zeros_like(u)
    with pytest.raises(L.PnopError) as e:
        ctx.pnop_gradient(u, -1.0, 0.05, g)
    assert e.value.code == -4
    ctx.close()


def test_hbm_budget_too_small_for_the_checkpoints(env):
    torch, L = env
    need = L.pnop_context_bytes(32, 16, 32, 10.0, 0, 4)
    with pytest.raises(L.PnopError) as e:
        _ctx(L, hbm=1 << 20)  # 1 MiB cannot hold the operators
    assert e.value.code == -2
    ctx = _ctx(L, hbm=need, snaps=1000)  # 1000 slots (350 MB) cannot fit in the budget
    u = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    u[2, 5, ctx.M, 0] = 1e-3
    with pytest.raises(L.PnopError) as e:
        ctx.pnop_gradient(u, -1.0, 10.0, torch.zeros_like(u))
    assert e.value.code == -2
    ctx.close()
