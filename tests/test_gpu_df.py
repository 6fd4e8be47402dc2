"""The double-FP32 option (PNOP_DF): the explicit banded products (curl,
divergence, pressure gradient and their transposes) in double-float
arithmetic, about 48 significant bits (Dekker 1971), everything else as in the
FP64 path.

* PNOP_DF against the FP64 oracle: each operator and the whole gradient at
  the FP64 tolerance, relative 1e-10 (double-float rounds at 2^-48, 32 times
  FP64's unit, which leaves these tests two orders of magnitude of room).
* PNOP_MIXED_DF (FP32 transforms as well): the mixed-precision budget, energy
  gain within 1e-5 and gradient cosine at least 0.99999, against the oracle on
  the 200-step small workload's grid and against the FP64 GPU gradient at the
  full 64x64x256 grid.
"""
import math

import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

from tests.test_gpu_parity import Case, RAGGED, SMALL, dev, host, rel

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return _lib


@pytest.fixture(scope="module", params=["small", "ragged"])
def case(L, request):
    if request.param == "small":
        return Case(L, **SMALL, precision=L.PNOP_DF)
    return Case(L, **RAGGED, Wo=5.6, A=0.85, tau0=3.0, precision=L.PNOP_DF)


def test_df_operators_match_the_oracle(case, L):
    c = case
    u = c.field(3, 1e-2)
    nb = c.field(8, 1.0)
    F = c.field(6, 1e-1)
    t = c.tau0 + 0.37
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_CURL, dev(u), None, out)
    errs = {"curl": rel(host(out), c.o.curl(u))}
    c.ctx.pnop_apply(L.OP_NONLINEAR, dev(u), None, out, t)
    errs["nonlinear"] = rel(host(out), c.o.nonlinear(u, t))
    c.ctx.pnop_apply(L.OP_NONLINEAR_T, dev(u), dev(nb), out, t)
    errs["nonlinear_T"] = rel(host(out), c.o.nonlinearT(u, t, nb))
    c.ctx.pnop_apply(L.OP_STAGE, dev(u), dev(F), out)
    errs["stage"] = rel(host(out), c.o.stage(u, F))
    ref_u, ref_F = c.o.stageT(nb)
    c.ctx.pnop_apply(L.OP_STAGE_T_U, dev(nb), None, out)
    errs["stage_T_u"] = rel(host(out), ref_u)
    c.ctx.pnop_apply(L.OP_STAGE_T_F, dev(nb), None, out)
    errs["stage_T_F"] = rel(host(out), ref_F)
    print("double-FP32 operator errors:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) < TOL, errs


def test_df_steps_and_gradient_match_the_oracle(case, L):
    c = case
    u0 = c.field(16, 1e-3)
    x = dev(u0)
    c.ctx.pnop_step_forward(x, c.tau0, 12)
    assert rel(host(x), c.o.forward(u0, c.tau0, 12)) < TOL
    nsteps = 9
    ET, gref = c.o.gradient(u0, c.tau0, nsteps)
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, nsteps * c.o.p.dt, g)
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert rel(host(g), gref) < TOL


def test_df_cfg1_gradient(L):
    """The 200-step small workload (Nr=32, |m|<=7, |k|<=15) in PNOP_DF."""
    c = Case(L, nr=32, M=7, K=15, Lz=10.0, Re=2000.0, dt=0.01, Wo=8.0, A=1.0, snaps=16, precision=L.PNOP_DF)
    u0 = c.field(0, 1e-6)
    ET, gref = c.o.gradient(u0, 0.0, 200)
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, 2.0, g)
    e = rel(host(g), gref)
    print(f"double-FP32 200-step gradient: gain rel {abs(gain / (ET / c.o.energy(u0)) - 1):.2e}, max-norm rel {e:.2e}")
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert e < TOL


def test_mixed_df_budget_against_the_oracle(L):
    c = Case(L, nr=32, M=7, K=15, Lz=10.0, Re=2000.0, dt=0.01, precision=L.PNOP_MIXED_DF)
    u0 = c.field(0, 1e-6)
    ET, gref = c.o.gradient(u0, 0.0, 50)
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, 0.5, g)
    gh = host(g)
    cos = c.o.inner(gh, gref) / math.sqrt(c.o.inner(gh, gh) * c.o.inner(gref, gref))
    assert abs(gain / (ET / c.o.energy(u0)) - 1) <= 1e-5
    assert cos >= 0.99999


def test_mixed_df_budget_against_fp64_at_full_size(L):
    import torch
    NR, NTH, NZ, LZ, RE, WO, A, DT = 64, 64, 256, 100.0, 2000.0, 8.0, 1.0, 0.0025
    tau0 = 0.25 * 2 * math.pi * RE / WO ** 2
    out = {}
    for prec in (L.PNOP_FP64, L.PNOP_MIXED_DF):
        ctx = L.Context(NR, NTH, NZ, LZ, RE, DT, WO, A, tau0, prec, 4)
        r = np.array(ctx.pnop_grid_points())
        u = torch.from_numpy(synth.oblique_field(r, NTH // 2 - 1, NZ // 2 - 1, LZ, seed=0)).to("cuda")
        g = torch.zeros_like(u)
        gain = ctx.pnop_gradient(u, 1e-5, 12 * DT, g)
        out[prec] = (gain, g, ctx)
    (g64, d64, c64), (gdf, ddf, _) = out[L.PNOP_FP64], out[L.PNOP_MIXED_DF]
    cos = c64.pnop_inner(d64, ddf) / math.sqrt(c64.pnop_inner(d64, d64) * c64.pnop_inner(ddf, ddf))
    assert abs(gdf / g64 - 1) <= 1e-5
    assert cos >= 0.99999
    for v in out.values():
        v[2].close()
