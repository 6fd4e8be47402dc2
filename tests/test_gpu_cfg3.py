"""The torch.autograd.Function check at its stated size: the grid and physics
of the localised-perturbation workload (nr=48, |m|<=15, |k|<=47, Lz=50,
Re=2500, A=1, Wo=8, dt=0.005), horizon 5 (1000 steps).

* FinalEnergy's backward against central finite differences with step
  h = 1e-7 |u0| (FP64) along 16 seeded directions.
* FinalEnergy's backward over the first 100 steps against the oracle gradient
  (the stored oracle values of tests/golden/cfg2_oracle_100steps.json).
* Recompute versus store: snapshot budgets 4/8/16/64 give bitwise the same
  gradient, Eq. 2.18's forward-step counts, and device memory that grows by
  one field per added slot.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu

NR, M, K, LZ, RE, WO, A, DT = 48, 15, 47, 50.0, 2500.0, 8.0, 1.0, 0.005
E0, NSTEPS = 1e-5, 1000
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg2_oracle_100steps.json")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib, autograd
    o = po.Oracle(po.Params(nr=NR, M=M, K=K, Lz=LZ, Re=RE, dt=DT, Wo=WO, A=A))
    u0 = o.scale_to(synth.localised_field(o.r, M, K, LZ, seed=0), E0)
    return torch, _lib, autograd, o, u0


def context(L, snaps):
    return L.Context(NR, 2 * (M + 1), 2 * (K + 1), LZ, RE, DT, WO, A, 0.0, L.PNOP_FP64, snaps)


def backward(env, ctx, nsteps):
    torch, L, ag, o, u0 = env
    x = torch.from_numpy(u0).to("cuda").requires_grad_(True)
    E = ag.final_energy(x, ctx, nsteps * DT)
    E.backward()
    return E.item(), x.grad.detach().cpu().numpy()


def test_autograd_matches_central_differences_along_16_directions(env):
    torch, L, ag, o, u0 = env
    ctx = context(L, 16)
    ET, g = backward(env, ctx, NSTEPS)
    h = 1e-7 * math.sqrt(np.sum(np.abs(u0) ** 2))

    def energy(field):
        x = torch.from_numpy(field).to("cuda")
        ctx.pnop_step_forward(x, 0.0, NSTEPS)
        return ctx.pnop_energy(x)

    worst = 0.0
    for seed in range(1, 17):
        v = synth.localised_field(o.r, M, K, LZ, seed=300 + seed)
        v = v / math.sqrt(np.sum(np.abs(v) ** 2))
        Ep, Em = energy(u0 + h * v), energy(u0 - h * v)
        fd = (Ep - Em) / (2 * h)
        ad = float(np.sum(np.real(np.conj(g) * v)))
        # rounding floor of the difference: E(T) to within 100 units in the last place
        floor = 100 * np.finfo(np.float64).eps * (abs(Ep) + abs(Em)) / (2 * h)
        worst = max(worst, abs(fd - ad) / abs(ad))
        assert abs(fd - ad) <= 1e-6 * abs(ad) + floor, (seed, fd, ad, floor)
    print(f"cfg3 FD check: E(T)/E0 = {ET / E0:.9g}, worst relative FD gap {worst:.3e}")
    ctx.close()


def test_autograd_first_100_steps_match_the_oracle(env):
    torch, L, ag, o, u0 = env
    ref = json.load(open(GOLDEN))
    assert ref["nsteps"] == 100 and ref["E0"] == E0
    ctx = context(L, 8)
    ET, ge = backward(env, ctx, 100)
    g = ge / o.What[None]                       # Euclidean gradient -> Riesz representer
    assert abs(ET / E0 / ref["gain"] - 1) < 1e-10
    err = max(abs(g[tuple(i)] - complex(*z)) for i, z in ref["samples"])
    tol = max(1e-10, 2 * ref["oracle_spread"]["grad_maxnorm_rel"])  # as in the cfg-2 parity test
    assert err <= tol * ref["grad_max"]
    n2 = o.inner(g, g)
    for seed, dot in zip(ref["dir_seeds"], ref["grad_dot_dirs"]):
        v = synth.random_field(o.r, M, K, LZ, seed=seed)
        assert abs(o.inner(g, v) - dot) <= 1e-10 * math.sqrt(n2 * o.inner(v, v)), seed
    ctx.close()


def test_snapshot_budget_sweep_store_versus_recompute(env):
    torch, L, ag, o, u0 = env
    grads, advs, nbytes = [], [], []
    for s in (4, 8, 16, 64):
        ctx = context(L, s)
        _, g = backward(env, ctx, NSTEPS)
        adv, nadj, _ = ctx.pnop_gradient_stats()
        assert nadj == NSTEPS
        assert adv == po.revolve_advances(NSTEPS, s) + 1
        grads.append(g)
        advs.append(adv)
        nbytes.append(ctx.pnop_device_bytes())
        ctx.close()
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])
    field = 3 * NR * (2 * M + 1) * (K + 1) * 16
    for (s1, b1), (s2, b2) in zip(zip((4, 8, 16, 64), nbytes), zip((8, 16, 64), nbytes[1:])):
        assert b2 - b1 == (s2 - s1) * field, (s1, s2, b1, b2)
    print("cfg3 budget sweep (slots, forward steps, device MB):",
          [(s, a, round(b / 2 ** 20, 1)) for s, a, b in zip((4, 8, 16, 64), advs, nbytes)])
