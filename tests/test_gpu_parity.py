"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerance for the FP64 path: relative 1e-10 (max-norm of
the difference over the max-norm of the oracle result); mixed precision:
energy-gain relative error <= 1e-5 and gradient cosine >= 0.99999.
"""
import math

import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

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


def torch_mod():
    import torch
    return torch


def dev(x):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


class Case:
    def __init__(self, L, nr, M, K, Lz, Re, dt, Wo=8.0, A=1.0, tau0=0.0, precision=0, snaps=8):
        self.ctx = L.Context(nr, 2 * (M + 1), 2 * (K + 1), Lz, Re, dt, Wo, A, tau0, precision, snaps)
        self.o = po.Oracle(po.Params(nr=nr, M=M, K=K, Lz=Lz, Re=Re, dt=dt, Wo=Wo, A=A))
        self.tau0 = tau0

    def field(self, seed, E0, kind="random"):
        o = self.o
        p = o.p
        if kind == "random":
            u = synth.random_field(o.r, p.M, p.K, p.Lz, seed=seed)
        elif kind == "localised":
            u = synth.localised_field(o.r, p.M, p.K, p.Lz, seed=seed)
        else:
            raise ValueError(kind)
        return o.scale_to(u, E0)

    def zeros(self):
        return dev(np.zeros(self.ctx.shape, np.complex128))


SMALL = dict(nr=12, M=3, K=5, Lz=10.0, Re=2000.0, dt=0.01)
# ragged: 3(M+1) = 27 (radix-3 only), nk = 18 (two k tiles, ragged tail), odd nr
RAGGED = dict(nr=11, M=8, K=17, Lz=7.0, Re=1500.0, dt=0.005)


@pytest.fixture(scope="module")
def small(L):
    return Case(L, **SMALL)


@pytest.fixture(scope="module")
def ragged(L):
    return Case(L, **RAGGED, Wo=5.6, A=0.85, tau0=3.0)


# Lengths served by the two-pass register FFT kernels (N = N1 N2): theta and z
# at 96 (8 x 12), z at 384 (16 x 24) with theta at 24 (Stockham), theta and z
# at 192 (16 x 12).
TWO_PASS = {
    "tp96": dict(nr=10, M=31, K=31, Lz=9.0, Re=1800.0, dt=0.004),
    "tp384": dict(nr=10, M=7, K=127, Lz=40.0, Re=1800.0, dt=0.004),
    "tp192": dict(nr=10, M=63, K=63, Lz=20.0, Re=1800.0, dt=0.004),
}


@pytest.fixture(scope="module", params=sorted(TWO_PASS))
def two_pass(L, request):
    return Case(L, **TWO_PASS[request.param], Wo=6.0, A=0.9, tau0=0.5)


@pytest.fixture(scope="module")
def two_pass_mixed(L, two_pass):
    prm = {k: getattr(two_pass.o.p, k) for k in ("nr", "M", "K", "Lz", "Re", "dt")}
    c = Case(L, **prm, Wo=6.0, A=0.9, tau0=0.5, precision=1)
    c.o = two_pass.o
    return c


def test_two_pass_transforms_nonlinear(two_pass, two_pass_mixed, L):
    c = two_pass
    u = c.field(21, 1e-2)
    nb = c.field(22, 1.0)
    t = c.tau0 + 0.41
    ref = c.o.nonlinear(u, t)
    refT = c.o.nonlinearT(u, t, nb)
    for cc, tol in ((c, 1e-12), (two_pass_mixed, 1e-5)):
        out = cc.zeros()
        cc.ctx.pnop_apply(L.OP_NONLINEAR, dev(u), None, out, t)
        assert rel(host(out), ref) < tol
        cc.ctx.pnop_apply(L.OP_NONLINEAR_T, dev(u), dev(nb), out, t)
        assert rel(host(out), refT) < tol


def test_two_pass_forward_step(two_pass):
    c = two_pass
    u0 = c.field(23, 1e-2)
    x = dev(u0)
    c.ctx.pnop_step_forward(x, c.tau0, 1)
    assert rel(host(x), c.o.forward(u0, c.tau0, 1)) < TOL


def test_wide_radial_grid_uses_the_shared_memory_solver(L):
    """More radial points than the register-resident solver holds (64): the
    shared-memory banded solver runs instead.  Steps, the adjoint step and a
    gradient against the oracle at nr = 72."""
    c = Case(L, nr=72, M=2, K=3, Lz=8.0, Re=1500.0, dt=0.005, Wo=6.0, A=0.7, tau0=1.0, snaps=3)
    u0 = c.field(41, 1e-2)
    x = dev(u0)
    c.ctx.pnop_step_forward(x, c.tau0, 3)
    assert rel(host(x), c.o.forward(u0, c.tau0, 3)) < TOL
    lam = c.field(42, 1.0)
    y = dev(lam)
    c.ctx.pnop_step_adjoint(dev(u0), y, c.tau0)
    W = c.o.What[None]
    assert rel(host(y), c.o.adjoint_step(u0, c.tau0, W * lam) / W) < TOL
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, 4 * c.o.p.dt, g)
    ET, gref = c.o.gradient(u0, c.tau0, 4)
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert rel(host(g), gref) < TOL


def test_grid_points_match(small):
    np.testing.assert_allclose(small.ctx.pnop_grid_points(), small.o.r, rtol=0, atol=1e-15)


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_energy_and_inner(case, request):
    c = request.getfixturevalue(case)
    a = c.field(1, 1e-3)
    b = c.field(2, 1e-3)
    assert abs(c.ctx.pnop_energy(dev(a)) / c.o.energy(a) - 1) < 1e-13
    assert abs(c.ctx.pnop_inner(dev(a), dev(b)) - c.o.inner(a, b)) < 1e-13 * math.sqrt(c.o.inner(a, a) * c.o.inner(b, b))


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_curl(case, request, L):
    c = request.getfixturevalue(case)
    u = c.field(3, 1e-2)
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_CURL, dev(u), None, out)
    assert rel(host(out), c.o.curl(u)) < 1e-12


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_nonlinear_term(case, request, L):
    c = request.getfixturevalue(case)
    u = c.field(4, 1e-2)
    t = c.tau0 + 0.37
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_NONLINEAR, dev(u), None, out, t)
    assert rel(host(out), c.o.nonlinear(u, t)) < 1e-12


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_stage_map(case, request, L):
    c = request.getfixturevalue(case)
    u = c.field(5, 1e-2)
    F = c.field(6, 1e-1)
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_STAGE, dev(u), dev(F), out)
    assert rel(host(out), c.o.stage(u, F)) < 1e-11


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_nonlinear_transpose(case, request, L):
    c = request.getfixturevalue(case)
    u = c.field(7, 1e-2)
    nb = c.field(8, 1.0)
    t = c.tau0 + 1.1
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_NONLINEAR_T, dev(u), dev(nb), out, t)
    assert rel(host(out), c.o.nonlinearT(u, t, nb)) < 1e-12


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_stage_transposes(case, request, L):
    c = request.getfixturevalue(case)
    ub = c.field(9, 1.0)
    ref_u, ref_F = c.o.stageT(ub)
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_STAGE_T_U, dev(ub), None, out)
    assert rel(host(out), ref_u) < 1e-11
    c.ctx.pnop_apply(L.OP_STAGE_T_F, dev(ub), None, out)
    assert rel(host(out), ref_F) < 1e-11


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_mode_energy_spectrum(case, request):
    c = request.getfixturevalue(case)
    u = c.field(15, 1e-3)
    got = c.ctx.pnop_mode_energy(dev(u))
    ref = c.o.mode_energy(u)
    assert np.abs(got - ref).max() <= 1e-13 * ref.sum()


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_resolution_measures(case, request):
    """pnop_resolution (device reduction) against Oracle.resolution: e_M and
    e_K relative 1e-12, with a given E0 and with the field's own energy."""
    c = request.getfixturevalue(case)
    p = c.o.p
    u = c.o.scale_to(synth.random_field(c.o.r, p.M, p.K, p.Lz, seed=19, decay=1.5), 2e-3)
    for E0 in (1e-3, -1.0):
        eM, eK = c.ctx.pnop_resolution(dev(u), E0)
        rM, rK = c.o.resolution(u, E0 if E0 > 0 else c.o.energy(u))
        assert rM > 0 and rK > 0
        assert abs(eM / rM - 1) < 1e-12 and abs(eK / rK - 1) < 1e-12


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_admissible_projection(case, request, L):
    from oracle import adjoint_looping as al
    c = request.getfixturevalue(case)
    rng = np.random.default_rng(13)
    g = c.field(14, 1.0) + 0.1 * (rng.standard_normal(c.ctx.shape) + 1j * rng.standard_normal(c.ctx.shape))
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_PROJECT, dev(g), None, out)
    ref = al.project_admissible(c.o, g)
    assert rel(host(out), ref) < 1e-9
    assert np.abs(c.o.divergence(host(out))).max() < 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_forward_steps(case, request):
    c = request.getfixturevalue(case)
    u0 = c.field(10, 1e-2)
    x = dev(u0)
    n = 12
    c.ctx.pnop_step_forward(x, c.tau0, n)
    ref = c.o.forward(u0, c.tau0, n)
    assert rel(host(x), ref) < TOL


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_adjoint_step(case, request):
    c = request.getfixturevalue(case)
    u = c.field(11, 1e-2)
    lam = c.field(12, 1.0)
    t = c.tau0 + 0.2
    x = dev(lam)
    c.ctx.pnop_step_adjoint(dev(u), x, t)
    W = c.o.What[None]
    ref = c.o.adjoint_step(u, t, W * lam) / W
    assert rel(host(x), ref) < TOL


def test_adjoint_step_dot_product_through_abi(small):
    """<J v, w> = <v, J^+ w> with J v from the GPU forward (5-point, exact for the quartic step)."""
    c = small
    u = c.field(13, 1e-2)
    v = c.field(14, 1e-2)
    w = c.field(15, 1.0)
    t = 0.4

    def step(e):
        x = dev(u + e * v)
        c.ctx.pnop_step_forward(x, t, 1)
        return host(x)

    h = 1.0
    jv = (step(-2 * h) - 8 * step(-h) + 8 * step(h) - step(2 * h)) / (12 * h)
    x = dev(w)
    c.ctx.pnop_step_adjoint(dev(u), x, t)
    lhs = c.o.inner(jv, w)
    rhs = c.o.inner(v, host(x))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_gradient_and_budgets(case, request, L):
    c = request.getfixturevalue(case)
    u0 = c.field(16, 1e-3)
    nsteps = 9
    horizon = nsteps * c.o.p.dt
    ET, gref = c.o.gradient(u0, c.tau0, nsteps)
    E0 = c.o.energy(u0)
    grads = []
    for snaps in (1, 2, 3, 12):
        ctx = L.Context(c.o.p.nr, 2 * (c.o.p.M + 1), 2 * (c.o.p.K + 1), c.o.p.Lz, c.o.p.Re, c.o.p.dt, c.o.p.Wo,
                        c.o.p.A, c.tau0, 0, snaps)
        g = c.zeros()
        gain = ctx.pnop_gradient(dev(u0), -1.0, horizon, g)
        adv, nadj, _ = ctx.pnop_gradient_stats()
        assert nadj == nsteps
        assert adv == po.revolve_advances(nsteps, snaps) + 1   # + the step to the terminal state
        assert abs(gain / (ET / E0) - 1) < TOL
        assert rel(host(g), gref) < TOL
        grads.append(host(g))
        ctx.close()
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])  # recomputation is bitwise deterministic


def test_gradient_rescales_to_E0(small):
    c = small
    u0 = c.field(17, 1.0)
    E0 = 1e-4
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), E0, 5 * c.o.p.dt, g)
    us = c.o.scale_to(u0, E0)
    ET, gref = c.o.gradient(us, 0.0, 5)
    assert abs(gain / (ET / E0) - 1) < TOL
    assert rel(host(g), gref) < TOL


def test_gradient_host_buffers(small):
    c = small
    u0 = c.field(18, 1e-3)
    gh = np.zeros(c.ctx.shape, np.complex128)
    gain = c.ctx.pnop_gradient_host(np.ascontiguousarray(u0), -1.0, 4 * c.o.p.dt, gh)
    ET, gref = c.o.gradient(u0, 0.0, 4)
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert rel(gh, gref) < TOL


def test_cfg1_gradient_parity(L):
    """Nr=32, |m|<=7, |k|<=15 (24 x 48 physical), L=10, Re=2000, A=1, Wo=8,
    200 steps of dt=0.01, random solenoidal u0 at E0=1e-6."""
    c = Case(L, nr=32, M=7, K=15, Lz=10.0, Re=2000.0, dt=0.01, Wo=8.0, A=1.0, snaps=16)
    u0 = c.field(0, 1e-6)
    nsteps = 200
    ET, gref = c.o.gradient(u0, 0.0, nsteps)
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, nsteps * 0.01, g)
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert rel(host(g), gref) < TOL


def test_mixed_precision_error_budget(L):
    c = Case(L, nr=32, M=7, K=15, Lz=10.0, Re=2000.0, dt=0.01, precision=1)
    u0 = c.field(0, 1e-6)
    nsteps = 50
    ET, gref = c.o.gradient(u0, 0.0, nsteps)
    g = c.zeros()
    gain = c.ctx.pnop_gradient(dev(u0), -1.0, nsteps * 0.01, g)
    G = ET / c.o.energy(u0)
    gh = host(g)
    cos = c.o.inner(gh, gref) / math.sqrt(c.o.inner(gh, gh) * c.o.inner(gref, gref))
    assert abs(gain / G - 1) <= 1e-5
    assert cos >= 0.99999



@pytest.mark.parametrize("case", ["small", "ragged"])
def test_continuous_adjoint_forcing(case, request, L):
    c = request.getfixturevalue(case)
    u = c.field(31, 1e-2)
    w = c.field(32, 1.0)
    t = c.tau0 + 0.23
    out = c.zeros()
    c.ctx.pnop_apply(L.OP_NONLINEAR_ADJ, dev(u), dev(w), out, t)
    assert rel(host(out), c.o.nonlinear_adj(w, u, t)) < 1e-12


def test_continuous_adjoint_forcing_two_pass(two_pass, two_pass_mixed, L):
    c = two_pass
    u = c.field(33, 1e-2)
    w = c.field(34, 1.0)
    t = c.tau0 + 0.41
    ref = c.o.nonlinear_adj(w, u, t)
    for cc, tol in ((c, 1e-12), (two_pass_mixed, 1e-5)):
        out = cc.zeros()
        cc.ctx.pnop_apply(L.OP_NONLINEAR_ADJ, dev(u), dev(w), out, t)
        assert rel(host(out), ref) < tol


@pytest.mark.parametrize("case", ["small", "ragged"])
def test_continuous_adjoint_gradient(case, request, L):
    c = request.getfixturevalue(case)
    u0 = c.field(35, 1e-2)
    n = 8
    ET, gref = c.o.gradient_continuous(u0, c.tau0, n)
    g = c.zeros()
    gain = c.ctx.pnop_gradient_continuous(dev(u0), -1.0, n * c.o.p.dt, g)
    assert abs(gain / (ET / c.o.energy(u0)) - 1) < TOL
    assert rel(host(g), gref) < TOL


def test_continuous_adjoint_gradient_mixed_precision(L):
    c = Case(L, nr=32, M=7, K=15, Lz=10.0, Re=2000.0, dt=0.01, precision=1)
    u0 = c.field(0, 1e-6)
    n = 30
    ET, gref = c.o.gradient_continuous(u0, 0.0, n)
    g = c.zeros()
    gain = c.ctx.pnop_gradient_continuous(dev(u0), -1.0, n * 0.01, g)
    gh = host(g)
    cos = c.o.inner(gh, gref) / math.sqrt(c.o.inner(gh, gh) * c.o.inner(gref, gref))
    assert abs(gain / (ET / c.o.energy(u0)) - 1) <= 1e-5
    assert cos >= 0.99999
