"""The FP64-versus-mixed workload on a localised perturbation, at its stated
size: nr=48, |m|<=15, |k|<=47 (48 x 144 physical), Lz=50, Re=2500, A=1, Wo=8,
dt=0.005, horizon 20 (4000 steps), binomial checkpointing with 32 slots,
localised seed (Gaussian envelope of width 3 in z), E0=1e-5.

* The mixed-precision gradient (FP32 transforms and products, FP64 radial
  algebra and inner products) against the FP64 gradient over the whole
  4000-step horizon: energy-gain relative error <= 1e-5 and gradient cosine
  >= 0.99999, both in the energy inner product (Eq. 2.2).
* The FP64 gradient over the first 100 steps against the oracle's, relative
  1e-10.  The oracle needs minutes for that prefix, so its values are stored
  (tests/golden/cfg2_oracle_100steps.json, written by make_cfg2_oracle.py
  beside it, which calls only the oracle): the gain, the gradient's energy
  norm, its inner products with eight seeded directions and 320 sampled
  coefficients.  The coefficients are held to 1e-10 of the largest, or to
  twice the spread between two equally valid roundings of the oracle itself
  where that is larger (it is about 1e-10 here).
* The 4000-step sweep takes Eq. 2.18's number of forward steps plus one.
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
E0, NSTEPS, SNAPS = 1e-5, 4000, 32
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg2_oracle_100steps.json")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    o = po.Oracle(po.Params(nr=NR, M=M, K=K, Lz=LZ, Re=RE, dt=DT, Wo=WO, A=A))
    u0 = o.scale_to(synth.localised_field(o.r, M, K, LZ, seed=0), E0)
    return torch, _lib, o, u0


def gradient(env, precision, nsteps, snaps=SNAPS):
    torch, L, o, u0 = env
    ctx = L.Context(NR, 2 * (M + 1), 2 * (K + 1), LZ, RE, DT, WO, A, 0.0, precision, snaps)
    x = torch.from_numpy(u0).to("cuda")
    g = torch.zeros_like(x)
    gain = ctx.pnop_gradient(x, -1.0, nsteps * DT, g)
    stats = ctx.pnop_gradient_stats()
    return ctx, gain, g, stats


@pytest.fixture(scope="module")
def full_horizon(env):
    c64, gain64, g64, st64 = gradient(env, 0, NSTEPS)
    c32, gain32, g32, st32 = gradient(env, 1, NSTEPS)
    yield c64, gain64, g64, st64, gain32, g32, st32
    c64.close()
    c32.close()


def test_checkpointed_sweep_takes_eq_2_18_advances(full_horizon):
    st64, st32 = full_horizon[3], full_horizon[6]
    for adv, nadj, _ in (st64, st32):
        assert nadj == NSTEPS
        assert adv == po.revolve_advances(NSTEPS, SNAPS) + 1 == 11406


def test_mixed_precision_budget_over_4000_steps(full_horizon):
    c64, gain64, g64, _, gain32, g32, _ = full_horizon
    assert math.isfinite(gain64) and gain64 > 0
    rel_gain = abs(gain32 / gain64 - 1)
    cos = c64.pnop_inner(g32, g64) / math.sqrt(c64.pnop_inner(g32, g32) * c64.pnop_inner(g64, g64))
    print(f"cfg2 4000 steps: gain fp64 {gain64:.12g} mixed {gain32:.12g} rel {rel_gain:.3e} cos-1 {cos - 1:.3e}")
    assert rel_gain <= 1e-5
    assert cos >= 0.99999


def test_fp64_first_100_steps_match_the_oracle(env):
    torch, L, o, u0 = env
    ref = json.load(open(GOLDEN))
    assert ref["config"] == dict(nr=NR, M=M, K=K, Lz=LZ, Re=RE, dt=DT, Wo=WO, A=A)
    assert ref["E0"] == E0 and ref["nsteps"] == 100
    ctx, gain, g, _ = gradient(env, 0, 100, snaps=8)
    gh = g.cpu().numpy()
    assert abs(gain / ref["gain"] - 1) < 1e-10
    n2 = o.inner(gh, gh)
    assert abs(n2 / ref["grad_norm2"] - 1) < 1e-10
    for seed, dot in zip(ref["dir_seeds"], ref["grad_dot_dirs"]):
        v = synth.random_field(o.r, M, K, LZ, seed=seed)
        assert abs(o.inner(gh, v) - dot) <= 1e-10 * math.sqrt(n2 * o.inner(v, v)), seed
    # coefficient by coefficient: 1e-10 of the largest value, or twice the
    # spread of two equally valid oracle evaluations where that is larger (the
    # rounding floor of this 100-step, nr = 48 problem, recorded by the generator)
    err = max(abs(gh[tuple(i)] - complex(*z)) for i, z in ref["samples"])
    tol = max(1e-10, 2 * ref["oracle_spread"]["grad_maxnorm_rel"])
    print(f"cfg2 100-step FP64 vs oracle: max-norm {err / ref['grad_max']:.3e}, oracle spread"
          f" {ref['oracle_spread']['grad_maxnorm_rel']:.3e}")
    assert err <= tol * ref["grad_max"]
    ctx.close()
