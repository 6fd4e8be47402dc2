"""Pins of the adjoint-looping oracle (Section 2.3, Eq. 2.13-2.15).

* the roots lambda_+- of Eq. 2.14 keep the update on the energy shell, and real
  roots exist exactly up to alpha_max of Eq. 2.15 (closed form, any inner
  product);
* on a linear problem the loop converges to the exact optimum: the largest
  squared singular value of W^(1/2) J W^(-1/2), J the Jacobian of the
  N-step map at u = 0 assembled column by column, W the energy weights.
"""
import math

import numpy as np
import pytest

from oracle import adjoint_looping as al
from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth


def test_lambda_roots_keep_the_energy_shell():
    rng = np.random.default_rng(0)
    w = rng.uniform(0.5, 2.0, 40)
    inner = lambda a, b: float(np.sum(w * a * b))
    for trial in range(20):
        u = rng.standard_normal(40)
        ud = rng.standard_normal(40) + rng.uniform(-2, 2) * u
        E0 = 0.5 * inner(u, u)
        E0d = 0.5 * inner(ud, ud)
        C0 = inner(u, ud)
        amax = al.alpha_max(E0, E0d, C0)
        assert math.isfinite(amax) and amax > 0
        for a in (1e-3 * amax, 0.37 * amax, amax):
            for lam in al.lambda_pm(a, E0, E0d, C0):
                v = (1 + lam * a) * u - a * ud
                assert abs(0.5 * inner(v, v) / E0 - 1) < 1e-10
        lm, lp = al.lambda_pm(amax, E0, E0d, C0)
        assert abs(lp - lm) <= 1e-6 * max(1.0, abs(lp))
        a = 1.01 * amax  # beyond alpha_max the discriminant is negative
        b = (a * C0 - 2 * E0) / (2 * a * E0)
        assert b * b - (a * E0d - C0) / (a * E0) < 0
    # u_dagger parallel to u: the update cannot leave the ray, alpha_max is infinite
    u = rng.standard_normal(40)
    assert al.alpha_max(0.5 * inner(u, u), 0.5 * inner(3 * u, 3 * u), inner(u, 3 * u)) == math.inf


@pytest.fixture(scope="module")
def tiny():
    p = po.Params(nr=9, M=1, K=1, Lz=4.0, Re=500.0, dt=0.25, Wo=8.0, A=0.0)
    return po.Oracle(p), 20


def exact_linear_optimum(o, N, admissible=True):
    """max E(J u) / E(u) over u (in V when admissible), J the N-step map at
    u = 0 in real coordinates (real and imaginary parts of every entry)."""
    p = o.p
    shape = (3, p.nr, 2 * p.M + 1, p.K + 1)
    n = int(np.prod(shape))
    zero = np.zeros(shape, np.complex128)

    def basis(i):
        e = np.zeros(n, np.complex128)
        e[i % n] = 1.0 if i < n else 1j
        return e.reshape(shape)

    def real(x):
        return np.concatenate([x.real.ravel(), x.imag.ravel()])

    rows = []
    for i in range(2 * n):
        x = basis(i)
        for s in range(N - 1, -1, -1):
            x = o.adjoint_step(zero, s * p.dt, x)  # transpose of the linear step at u = 0
        rows.append(real(x))
    J = np.array(rows)  # row i of J is J^T e_i
    w = np.tile(np.broadcast_to(o.What[None], shape).ravel(), 2)
    Ms = np.sqrt(w)[:, None] * J / np.sqrt(w)[None, :]
    if admissible:
        # W^(1/2) P W^(-1/2) is an orthogonal projector; its unit eigenvectors span W^(1/2) V
        P = np.array([real(al.project_admissible(o, basis(i))) for i in range(2 * n)]).T
        Ps = np.sqrt(w)[:, None] * P / np.sqrt(w)[None, :]
        ev, Q = np.linalg.eigh(0.5 * (Ps + Ps.T))
        Ms = Ms @ Q[:, ev > 0.5]
    return np.linalg.svd(Ms, compute_uv=False)[0] ** 2


def test_admissible_projection_is_the_energy_orthogonal_projector(tiny):
    o, _ = tiny
    p = o.p
    rng = np.random.default_rng(2)
    shape = (3, p.nr, 2 * p.M + 1, p.K + 1)
    g = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    h = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Pg, Ph = al.project_admissible(o, g), al.project_admissible(o, h)
    scale = np.abs(g).max()
    assert np.abs(al.project_admissible(o, Pg) - Pg).max() < 1e-10 * scale       # idempotent
    assert np.abs(Pg[:, 0]).max() < 1e-12 * scale                                # no slip
    assert np.abs(o.divergence(Pg)).max() < 1e-9 * scale                         # solenoidal
    assert abs(o.inner(g - Pg, Ph)) < 1e-10 * math.sqrt(o.inner(g, g) * o.inner(h, h))  # orthogonal
    assert np.abs(Pg[:, :, ::-1, 0] - np.conj(Pg[:, :, :, 0])).max() < 1e-14 * scale  # Hermitian
    mean = Pg[:, :, p.M, 0]
    assert np.abs(mean[0]).max() == 0.0 and abs(np.dot(o.W, mean[2])) < 1e-12 * scale  # u_r, flux


@pytest.fixture(scope="module")
def tiny_optimum(tiny):
    o, N = tiny
    return exact_linear_optimum(o, N)


def test_adjoint_looping_reaches_the_exact_linear_optimum(tiny, tiny_optimum):
    o, N = tiny
    Gopt = tiny_optimum
    assert Gopt < exact_linear_optimum(o, N, admissible=False)  # the subspace matters
    E0 = 1e-20  # linear regime: the nonlinear term is 1e-10 of the linear one
    u0 = synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=1)
    u, hist, info = al.optimise(o, u0, 0.0, N, E0, max_iter=40, tol=1e-10)
    assert info["converged"]
    assert abs(o.energy(u) / E0 - 1) < 1e-12
    assert all(b > a for a, b in zip(hist, hist[1:]))  # accepted updates only raise G
    assert hist[0] < 0.5 * Gopt
    assert abs(hist[-1] / Gopt - 1) < 1e-6


def test_shorter_first_step_reaches_the_same_linear_optimum(tiny, tiny_optimum):
    """A first trial step of half alpha_max (the conditioning choice the GPU
    parity test of the optimiser uses) changes the path, not the optimum."""
    o, N = tiny
    E0 = 1e-20
    u0 = synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=1)
    u, hist, info = al.optimise(o, u0, 0.0, N, E0, max_iter=60, tol=1e-10, alpha_frac=0.5)
    assert info["converged"]
    assert abs(o.energy(u) / E0 - 1) < 1e-12
    assert all(b > a for a, b in zip(hist, hist[1:]))
    assert abs(hist[-1] / tiny_optimum - 1) < 1e-6


def test_continuous_adjoint_looping_stays_below_the_exact_optimum(tiny, tiny_optimum):
    """With gradients from the continuous adjoint (Eq. 2.9-2.11) the loop still
    only accepts growth of the exactly evaluated G, so it climbs toward, and can
    never pass, the exact optimum; it stops where the approximate gradient
    (O(1) radial discretisation error on 9 points) no longer gives growth."""
    o, N = tiny
    E0 = 1e-20
    u0 = synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=1)
    u, hist, info = al.optimise(o, u0, 0.0, N, E0, max_iter=20, tol=1e-10, continuous=True)
    assert info["converged"]
    assert abs(o.energy(u) / E0 - 1) < 1e-12
    assert all(b > a for a, b in zip(hist, hist[1:]))
    assert hist[-1] <= tiny_optimum * (1 + 1e-10)
    assert hist[-1] > 0.95 * tiny_optimum > 1.9 * hist[0]
