"""Parity at the full 64x64x256 size in the launch configuration bench.py times
(nr=64, |m|<=31, |k|<=127, 96x384 physical, Lz=100, Re=2000, Wo=8, A=1,
dt=0.0025, tau0=T/4):

* sampled modes against the oracle, one by one, in the linear regime (a
  vanishing amplitude decouples the modes, so the oracle steps each sampled
  mode alone);
* properties that hold at any size: the adjoint dot-product identity through
  the C ABI, wall/flux/Hermitian invariants, bitwise determinism across
  checkpoint budgets, and the mixed-precision error budget against FP64.
"""
import math

import numpy as np
import pytest

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

pytestmark = pytest.mark.gpu

NR, NTH, NZ, LZ, RE, WO, A, DT = 64, 64, 256, 100.0, 2000.0, 8.0, 1.0, 0.0025
M, K = NTH // 2 - 1, NZ // 2 - 1
TAU0 = 0.25 * 2 * math.pi * RE / WO ** 2


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_10103_gb300 import build
    build.build()
    from paper_2509_10103_gb300 import _lib
    return torch, _lib


def ctx_for(L, precision, snaps=4):
    return L.Context(NR, NTH, NZ, LZ, RE, DT, WO, A, TAU0, precision, snaps)


def dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.fixture(scope="module")
def fields(env):
    torch, L = env
    c = ctx_for(L, L.PNOP_FP64)
    r = np.array(c.pnop_grid_points())
    c.close()
    u = synth.oblique_field(r, M, K, LZ, seed=0)
    v = synth.random_field(r, M, K, LZ, seed=5)
    w = synth.random_field(r, M, K, LZ, seed=6)
    return r, u, v, w


SAMPLE = [(0, 0), (1, 0), (-3, 5), (7, 80), (31, 127), (-31, 1), (16, 64), (-1, 80), (5, 0)]


def test_sampled_modes_match_the_oracle_in_the_linear_regime(env, fields):
    torch, L = env
    r = fields[0]
    o = po.Oracle(po.Params(nr=NR, M=M, K=K, Lz=LZ, Re=RE, dt=DT, Wo=WO, A=A))
    np.testing.assert_allclose(o.r, r, atol=1e-15)
    u = np.zeros((3, NR, 2 * M + 1, K + 1), np.complex128)
    for i, (m, k) in enumerate(SAMPLE):
        um = 1e-30 * synth.single_mode(r, m, k, LZ, seed=i)
        u[:, :, m + M, k] = um
        if k == 0 and m != 0:
            u[:, :, -m + M, 0] = np.conj(um)
    ctx = ctx_for(L, L.PNOP_FP64)
    x = dev(torch, u)
    ctx.pnop_step_forward(x, TAU0, 1)
    got = x.cpu().numpy()
    for (m, k) in SAMPLE:
        ref = o.linear_mode_step(u[:, :, m + M, k], m, k, TAU0)
        err = np.abs(got[:, :, m + M, k] - ref).max() / np.abs(ref).max()
        assert err < 1e-10, ((m, k), err)
    mask = np.zeros(got.shape[2:], bool)
    for (m, k) in SAMPLE:
        mask[m + M, k] = True
        if k == 0:
            mask[-m + M, 0] = True
    assert np.abs(got[:, :, ~mask]).max() < 1e-20 * np.abs(got).max()  # modes stay decoupled
    ctx.close()


def test_adjoint_dot_product_at_full_size(env, fields):
    torch, L = env
    _, u, v, w = fields
    ctx = ctx_for(L, L.PNOP_FP64)
    E = ctx.pnop_energy(dev(torch, u))
    u0 = u * math.sqrt(1e-5 / E)
    v = v * math.sqrt(1e-5 / ctx.pnop_energy(dev(torch, v)))

    def step(e):
        x = dev(torch, u0 + e * v)
        ctx.pnop_step_forward(x, TAU0, 1)
        return x

    h = 1.0
    jv = (step(-2 * h) - 8 * step(-h) + 8 * step(h) - step(2 * h)) / (12 * h)  # exact for the quartic step
    lam = dev(torch, w)
    ctx.pnop_step_adjoint(dev(torch, u0), lam, TAU0)
    lhs = ctx.pnop_inner(jv.contiguous(), dev(torch, w))
    rhs = ctx.pnop_inner(dev(torch, v), lam)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    ctx.close()


def test_step_invariants_at_full_size(env, fields):
    torch, L = env
    u = fields[1]
    for prec in (L.PNOP_FP64, L.PNOP_MIXED):
        ctx = ctx_for(L, prec)
        x = dev(torch, u * math.sqrt(1e-5 / ctx.pnop_energy(dev(torch, u))))
        ctx.pnop_step_forward(x, TAU0, 3)
        y = x.cpu().numpy()
        assert np.abs(y[:, 0]).max() == 0.0                                   # no-slip rows
        W = po.radial_weights(po.radial_grid(NR))
        assert abs(np.dot(W, y[2, :, M, 0])) < 1e-14 * np.abs(y).max()        # zero flux (Eq. 2.7)
        assert np.abs(y[:, :, ::-1, 0] - np.conj(y[:, :, :, 0])).max() < 1e-14 * np.abs(y).max()
        ctx.close()


def test_gradient_bitwise_across_budgets_and_mixed_error_budget(env, fields):
    torch, L = env
    u = fields[1]
    n = 12
    grads = {}
    for prec, snaps in ((L.PNOP_MIXED, 3), (L.PNOP_MIXED, 12), (L.PNOP_FP64, 4)):
        ctx = ctx_for(L, prec, snaps)
        g = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
        gain = ctx.pnop_gradient(dev(torch, u), 1e-5, n * DT, g)
        grads[(prec, snaps)] = (gain, g.cpu().numpy())
        ctx.close()
    gm3, gm12, gd = grads[(L.PNOP_MIXED, 3)], grads[(L.PNOP_MIXED, 12)], grads[(L.PNOP_FP64, 4)]
    assert gm3[0] == gm12[0] and np.array_equal(gm3[1], gm12[1])
    W = po.radial_weights(po.radial_grid(NR))
    wh = (2 * math.pi * LZ) * W[:, None, None] * np.where(np.arange(K + 1) == 0, 1.0, 2.0)[None, None, :]
    ip = lambda a, b: float(np.sum(wh[None] * np.real(np.conj(a) * b)))
    cos = ip(gm3[1], gd[1]) / math.sqrt(ip(gm3[1], gm3[1]) * ip(gd[1], gd[1]))
    assert abs(gm3[0] / gd[0] - 1) <= 1e-5
    assert cos >= 0.99999


@pytest.fixture(scope="module")
def nonlinear_ref(env, fields):
    """The oracle's N(u) and N'(u)^T nb at the full grid (a few einsums over the
    exact DFT matrices: seconds in numpy), u and nb with every mode excited."""
    torch, L = env
    r, _, v, w = fields
    o = po.Oracle(po.Params(nr=NR, M=M, K=K, Lz=LZ, Re=RE, dt=DT, Wo=WO, A=A))
    u = o.scale_to(v, 1.0)
    nb = o.scale_to(w, 1.0)
    t = TAU0 + 0.37
    return u, nb, t, o.nonlinear(u, t), o.nonlinearT(u, t, nb)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_nonlinear_term_and_transpose_match_the_oracle_at_full_size(env, nonlinear_ref, precision, tol):
    """OP_NONLINEAR and OP_NONLINEAR_T through the two-pass 96- and 384-point
    transform kernels the bench times, element by element against the oracle
    (max-norm relative).  FP64: 1e-10.  Mixed: FP32 transforms of lengths 96
    and 384 round each of their ~log2 N butterfly levels at 2^-24, about 1e-6
    of the largest value; 1e-5 leaves a factor 10 over that."""
    torch, L = env
    u, nb, t, ref, refT = nonlinear_ref
    ctx = ctx_for(L, precision)
    out = torch.zeros(ctx.shape, dtype=torch.complex128, device="cuda")
    ctx.pnop_apply(L.OP_NONLINEAR, dev(torch, u), None, out, t)
    e1 = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    ctx.pnop_apply(L.OP_NONLINEAR_T, dev(torch, u), dev(torch, nb), out, t)
    e2 = np.abs(out.cpu().numpy() - refT).max() / np.abs(refT).max()
    ctx.close()
    assert e1 < tol and e2 < tol, (e1, e2)
