"""Validation against a number the paper prints (Appendix A.1): in steady pipe
flow at Re = 1750, Lz = pi, the optimal perturbation for tau = 80 is the pair of
streamwise vortices (m = 1, k = 0), whose energy peaks at G_max ~ 219 near
t = 85.  Linear regime (E0 = 1e-20), adjoint looping through pnop_optimise,
Nr = 38, dt = 0.01, 8000 steps per sweep.  About a minute of GPU time, so it
runs only when PNOP_VALIDATION=1."""
import math
import os

import numpy as np
import pytest

from paper_2509_10103_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("PNOP_VALIDATION") != "1", reason="set PNOP_VALIDATION=1")]


def test_linear_optimum_steady_pipe_re1750():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib as L
    nr, M, K, Lz, Re, dt = 38, 2, 1, math.pi, 1750.0, 0.01
    ctx = L.Context(nr, 2 * (M + 1), 2 * (K + 1), Lz, Re, dt, 8.0, 0.0, 0.0, L.PNOP_FP64, 200)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(synth.random_field(r, M, K, Lz, seed=3)).to("cuda")
    stats, hist = ctx.pnop_optimise(u, 1e-20, 80.0, 40, 1e-8)
    print("optimise", stats, hist)
    # growth curve of the optimum: G(t) every 0.05 up to t = 100
    x = u.clone()
    E0 = ctx.pnop_energy(x)
    best, tbest = 0.0, 0.0
    for n in range(1, 2001):
        ctx.pnop_step_forward(x, (n - 1) * 5 * dt, 5)
        G = ctx.pnop_energy(x) / E0
        if G > best:
            best, tbest = G, n * 5 * dt
    print(f"G(80) = {stats['gain']:.3f}, G_max = {best:.3f} at t = {tbest:.2f}")
    energy_by_mode = [float((u[:, :, i, k].abs() ** 2).sum()) for i in range(2 * M + 1) for k in range(K + 1)]
    dominant = int(np.argmax(energy_by_mode))
    assert dominant // (K + 1) in (M - 1, M + 1) and dominant % (K + 1) == 0  # m = +-1, k = 0
    assert abs(best / 219.0 - 1) < 0.02
    assert abs(tbest - 85.05) < 2.0
    ctx.close()
