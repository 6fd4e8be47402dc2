"""Validation against numbers the paper prints (Appendix A), linear regime
(E0 = 1e-20), adjoint looping through pnop_optimise, Nr = 38, dt = 0.01.

* Appendix A.1: in steady pipe flow at Re = 1750, Lz = pi, the optimal
  perturbation for tau = 80 is the pair of streamwise vortices (m = 1, k = 0),
  whose energy peaks at G_max ~ 219 near t = 85.
* Appendix A.2: in pulsatile flow at Re = 2000, A = 1, Wo = 2, Lz = 10, with
  the perturbation introduced at tau0 = T/2 and optimised for tau = 0.02 T, the
  optimum is again the pair of streamwise vortices and its growth peaks at
  t ~ 90, i.e. 0.029 T (T = 2 pi Re / Wo^2 in these units).

Every checkpoint is kept (store-all: the states of these small grids take
under 200 MB), so each optimisation iteration costs one forward and one
adjoint sweep, and the loop stops once the gain changes by less than 1e-6
between iterations: about a minute of GPU time each."""
import math

import numpy as np
import pytest

from paper_2509_10103_gb300 import synth

from tests.test_oracle_pins import paper_numbers

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_linear_optimum_steady_pipe_re1750():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib as L
    nr, M, K, Lz, Re, dt = 38, 2, 1, math.pi, 1750.0, 0.01
    ctx = L.Context(nr, 2 * (M + 1), 2 * (K + 1), Lz, Re, dt, 8.0, 0.0, 0.0, L.PNOP_FP64, 8001)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(synth.random_field(r, M, K, Lz, seed=3)).to("cuda")
    stats, hist = ctx.pnop_optimise(u, 1e-20, 80.0, 25, 1e-6)
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
    P = paper_numbers()
    assert abs(best / P["steady_re1750_lzpi_tau80_Gmax"] - 1) < 0.02
    assert abs(tbest - P["steady_re1750_lzpi_tau80_tmax"]) < 2.0
    ctx.close()


def test_linear_optimum_pulsatile_wo2_peaks_at_0029T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib as L
    nr, M, K, Lz, Re, dt, Wo, A = 38, 2, 2, 10.0, 2000.0, 0.01, 2.0, 1.0
    T = 2 * math.pi * Re / Wo ** 2
    tau0, nsteps = T / 2, int(round(0.02 * T / dt))
    ctx = L.Context(nr, 2 * (M + 1), 2 * (K + 1), Lz, Re, dt, Wo, A, tau0, L.PNOP_FP64, nsteps + 1)
    r = np.array(ctx.pnop_grid_points())
    u = torch.from_numpy(synth.random_field(r, M, K, Lz, seed=3)).to("cuda")
    stats, hist = ctx.pnop_optimise(u, 1e-20, nsteps * dt, 20, 1e-6)
    print("optimise", stats, hist)
    x = u.clone()
    E0 = ctx.pnop_energy(x)
    best, tbest = 0.0, 0.0
    for n in range(1, 1501):  # growth curve every 0.1 up to t = 150
        ctx.pnop_step_forward(x, tau0 + (n - 1) * 10 * dt, 10)
        G = ctx.pnop_energy(x) / E0
        if G > best:
            best, tbest = G, n * 10 * dt
    print(f"G(tau) = {stats['gain']:.3f}, G_max = {best:.3f} at t = {tbest:.2f} = {tbest / T:.4f} T")
    e = ctx.pnop_mode_energy(u).sum(axis=0)
    e = e / e.sum()
    assert e[M - 1, 0] + e[M + 1, 0] > 0.99  # streamwise vortices: m = +-1, k = 0
    P = paper_numbers()
    assert abs(tbest - P["wo2_re2000_a1_lz10_tpeak"]) < 3.0
    assert abs(tbest / T - P["wo2_re2000_a1_lz10_tpeak_over_T"]) < 0.001
    assert stats["gain"] < best  # the growth goes on past the optimisation time
    ctx.close()
