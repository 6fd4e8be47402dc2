"""The autograd.Function wrapper: gradient against the oracle, against central
finite differences along seeded directions, and across checkpoint budgets
(store-all versus recomputation)."""
import math

import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib, autograd
    return torch, _lib, autograd


GRID = dict(nr=16, M=3, K=7, Lz=10.0, Re=2000.0, dt=0.01, Wo=8.0, A=1.0)


def _setup(env, snaps, nsteps=20, E0=1e-3, seed=3):
    torch, L, ag = env
    p = GRID
    ctx = L.Context(p["nr"], 2 * (p["M"] + 1), 2 * (p["K"] + 1), p["Lz"], p["Re"], p["dt"], p["Wo"], p["A"], 0.0, 0,
                    snaps)
    o = po.Oracle(po.Params(**p))
    u0 = o.scale_to(synth.random_field(o.r, p["M"], p["K"], p["Lz"], seed=seed), E0)
    return torch, L, ag, ctx, o, u0, nsteps


def test_autograd_gradient_matches_oracle(env):
    torch, L, ag, ctx, o, u0, n = _setup(env, snaps=4)
    x = torch.from_numpy(u0).to("cuda").requires_grad_(True)
    E = ag.final_energy(x, ctx, n * o.p.dt)
    (3.0 * E).backward()
    ET, g = o.gradient(u0, 0.0, n)
    assert abs(E.item() / ET - 1) < 1e-10
    ref = 3.0 * o.What[None] * g            # Euclidean gradient of 3 E
    got = x.grad.detach().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_autograd_gradient_matches_central_differences_along_16_directions(env):
    torch, L, ag, ctx, o, u0, n = _setup(env, snaps=4, nsteps=30)
    x = torch.from_numpy(u0).to("cuda").requires_grad_(True)
    E = ag.final_energy(x, ctx, n * o.p.dt)
    E.backward()
    g = x.grad.detach().cpu().numpy()
    scale = math.sqrt(np.sum(np.abs(u0) ** 2))
    for seed in range(1, 17):
        v = synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=100 + seed)
        v = v / math.sqrt(np.sum(np.abs(v) ** 2))
        h = 1e-7 * scale
        with torch.no_grad():
            Ep = ag.final_energy(torch.from_numpy(u0 + h * v).to("cuda"), ctx, n * o.p.dt).item()
            Em = ag.final_energy(torch.from_numpy(u0 - h * v).to("cuda"), ctx, n * o.p.dt).item()
        fd = (Ep - Em) / (2 * h)
        ad = float(np.sum(np.real(np.conj(g) * v)))
        assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-9 * np.abs(g).max(), (seed, fd, ad)


@pytest.mark.parametrize("budgets", [(4, 8, 16, 64, 0)])
def test_checkpoint_budgets_store_versus_recompute(env, budgets):
    torch = env[0]
    grads, stats = [], []
    for s in budgets:
        _, L, ag, ctx, o, u0, n = _setup(env, snaps=s, nsteps=48)
        x = torch.from_numpy(u0).to("cuda").requires_grad_(True)
        ag.final_energy(x, ctx, n * o.p.dt).backward()
        grads.append(x.grad.detach().cpu().numpy())
        adv, nadj, stores = ctx.pnop_gradient_stats()
        slots = min(s, n) if s > 0 else n      # budget 0: sized to memory, at most store-all
        assert nadj == n
        assert adv == po.revolve_advances(n, slots) + 1
        stats.append(adv)
        ctx.close()
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])
    assert stats == sorted(stats, reverse=True)  # more memory, fewer recomputations


def test_backward_without_forward_is_rejected(env):
    torch, L, ag, ctx, o, u0, n = _setup(env, snaps=2)
    g = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.PnopError):
        ctx.pnop_gradient_backward(1.0, g)
    ctx.pnop_gradient_forward(torch.from_numpy(u0).to("cuda"), -1.0, n * o.p.dt)
    ctx.pnop_step_forward(torch.from_numpy(u0).to("cuda"), 0.0, 1)  # discards the pending sweep
    with pytest.raises(L.PnopError):
        ctx.pnop_gradient_backward(1.0, g)
