"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each pin is chosen so that a plausible slip in the oracle (dropped term, wrong
sign or index, transposed operand, missing Hermitian factor) fails at least one
of them.  None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _zeros():
    z = {}
    with open(os.path.join(GOLDEN, "bessel_zeros.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, v = line.split()
            z[int(n)] = float(v)
    return z


def _oracle(**kw):
    d = dict(nr=12, M=2, K=3, Lz=10.0, Re=2000.0, dt=0.01, Wo=8.0, A=1.0)
    d.update(kw)
    return po.Oracle(po.Params(**d))


def _field(o, seed, E0):
    p = o.p
    return o.scale_to(synth.random_field(o.r, p.M, p.K, p.Lz, seed=seed), E0)


# ---------------------------------------------------------------- grid / quadrature
def test_radial_grid_is_half_chebyshev_lobatto():
    for nr in (8, 32, 64):
        r = po.radial_grid(nr)
        full = np.cos(np.pi * np.arange(2 * nr) / (2 * nr - 1))
        assert r[0] == 1.0 and np.all(np.diff(r) < 0) and r[-1] > 0
        np.testing.assert_allclose(np.concatenate([r, -r[::-1]]), full, atol=1e-15)


@pytest.mark.parametrize("nr", [8, 16, 32, 48, 64, 96, 128])
def test_quadrature_exact_on_even_polynomials_and_positive(nr):
    r = po.radial_grid(nr)
    W = po.radial_weights(r)
    assert np.all(W > 0)
    for i in range(nr):
        assert abs(np.dot(W, r ** (2 * i)) - 1.0 / (2 * i + 2)) < 1e-13


# ---------------------------------------------------------------- finite differences
@pytest.mark.parametrize("parity", [1, -1])
def test_fd_exact_on_parity_polynomials(parity):
    r = po.radial_grid(16)
    d1, d2 = po.fd_matrices(r, parity)
    first = 0 if parity == 1 else 1
    for p in range(first, 9, 2):  # degree <= 8 is inside the 9-point span
        f = r ** p
        df = p * r ** (p - 1) if p >= 1 else 0 * r
        ddf = p * (p - 1) * r ** (p - 2) if p >= 2 else 0 * r
        np.testing.assert_allclose(d1 @ f, df, atol=1e-9 * max(1, p))
        np.testing.assert_allclose(d2 @ f, ddf, atol=1e-7 * max(1, p * p))


def test_fd_converges_at_high_order():
    errs = []
    for nr in (16, 32):
        r = po.radial_grid(nr)
        d1, d2 = po.fd_matrices(r, 1)
        f = sp.jv(0, 3.0 * r)          # even function
        ddf = -9.0 * (sp.jv(0, 3 * r) - sp.jv(1, 3 * r) / (3 * r))  # J0'' at 3r
        errs.append(np.abs(d2 @ f - ddf).max())
    assert errs[1] < errs[0] / 2 ** 6


# ---------------------------------------------------------------- base flow
def test_bessel_series_matches_library():
    z = np.exp(0.75j * np.pi) * np.linspace(0.0, 18.0, 37)
    for nu in (0, 1):
        ref = sp.jv(nu, z)
        got = po.bessel_j(nu, z)
        assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(1.0, np.abs(ref)))


def test_womersley_steady_limit_and_no_slip():
    r = po.radial_grid(24)
    U, dU = po.womersley(r, 3.7, 2000.0, 8.0, 0.0)
    np.testing.assert_allclose(U, 1 - r ** 2, atol=0)
    U, dU = po.womersley(r, 3.7, 2000.0, 8.0, 1.0)
    assert abs(U[0]) < 1e-12


@pytest.mark.parametrize("Wo", [2.0, 8.0, 18.0])
def test_womersley_bulk_velocity_follows_ub(Wo):
    Re, A = 2000.0, 1.0
    r = po.radial_grid(64)
    W = po.radial_weights(r)
    T = 2 * np.pi * Re / Wo ** 2
    for t in np.linspace(0, T, 7):
        U, _ = po.womersley(r, t, Re, Wo, A)
        ub = 0.5 * (1 + A * np.sin(2 * np.pi * t / T))
        assert abs(2 * np.dot(W, U) - ub) < 1e-9


def test_womersley_quasi_steady_limit():
    r = po.radial_grid(24)
    Re, A, Wo = 2000.0, 0.7, 1e-3
    om = Wo ** 2 / Re
    for t in (0.0, 1e9, 2.3e9):
        U, dU = po.womersley(r, t, Re, Wo, A)
        np.testing.assert_allclose(U, (1 - r ** 2) * (1 + A * np.sin(om * t)), atol=1e-6)
        np.testing.assert_allclose(dU, -2 * r * (1 + A * np.sin(om * t)), atol=1e-6)


def test_womersley_solves_unsteady_stokes():
    # dU/dt - (U'' + U'/r)/Re must be uniform in r (the imposed pressure gradient)
    Re, Wo, A = 2000.0, 8.0, 1.0
    r = po.radial_grid(48)
    d1, d2 = po.fd_matrices(r, 1)
    t, h = 5.0, 1e-3
    Up, _ = po.womersley(r, t + h, Re, Wo, A)
    Um, _ = po.womersley(r, t - h, Re, Wo, A)
    U, dU = po.womersley(r, t, Re, Wo, A)
    np.testing.assert_allclose(d1 @ U, dU, atol=1e-7)
    g = (Up - Um) / (2 * h) - (d2 @ U + (d1 @ U) / r) / Re
    assert np.ptp(g[1:]) < 1e-5 * np.abs(dU).max()


# ---------------------------------------------------------------- transforms / products
def test_synth_matches_library_irfft():
    o = _oracle(M=3, K=4)
    u = _field(o, 3, 1.0)
    f = o.synth(u[2])
    p = o.p
    for j in (0, 5):
        full = np.zeros((o.ntheta, o.nz), np.complex128)
        for i, m in enumerate(o.m):
            full[m % o.ntheta, : p.K + 1] = u[2, j, i, :]
        ref = np.fft.irfft(np.fft.ifft(full, axis=0) * o.ntheta, n=o.nz, axis=1) * o.nz
        np.testing.assert_allclose(f[j], ref, atol=1e-13 * np.abs(ref).max())


def test_analysis_inverts_synth():
    o = _oracle(M=3, K=4)
    u = _field(o, 4, 1.0)
    np.testing.assert_allclose(o.analysis(o.synth(u[0])), u[0], atol=1e-14 * np.abs(u).max())


def test_nonlinear_term_is_energy_neutral():
    o = _oracle(M=3, K=4)
    u = _field(o, 5, 1e-2)
    w = o.curl(u)
    up = np.stack([o.synth(c) for c in u])
    wp = np.stack([o.synth(c) for c in w])
    nl = np.stack([o.analysis(c) for c in np.cross(up, wp, axis=0)])
    assert np.abs(nl).max() > 1e-4
    assert abs(o.inner(u, nl)) <= 1e-13 * math.sqrt(o.inner(u, u) * o.inner(nl, nl))


# ---------------------------------------------------------------- linear Stokes dynamics
def _decay_rate(o, u, n):
    E0 = o.energy(u)
    uN = o.forward(u, 0.0, n)
    return -math.log(o.energy(uN) / E0) / (2 * n * o.p.dt)


def _cn_rate(lam, Re, dt):
    a = lam * lam / Re
    return -math.log((1 - dt * a / 2) / (1 + dt * a / 2)) / dt


def test_stokes_mode_decay_rates():
    z = _zeros()
    o = _oracle(nr=32, M=1, K=1, Re=100.0, base=False)
    nr = o.p.nr
    # u_theta of (0,0) ~ J1(j11 r): rate j11^2/Re
    u = np.zeros((3, nr, 3, 2), complex)
    u[1, :, 1, 0] = 1e-8 * sp.jv(1, z[1] * o.r)
    assert abs(_decay_rate(o, u, 40) / _cn_rate(z[1], 100.0, o.p.dt) - 1) < 1e-7
    # flux-constrained u_z of (0,0) ~ J0(j21 r) - J0(j21): rate j21^2/Re
    u = np.zeros((3, nr, 3, 2), complex)
    u[2, :, 1, 0] = 1e-8 * (sp.jv(0, z[2] * o.r) - sp.jv(0, z[2]))
    assert abs(_decay_rate(o, u, 40) / _cn_rate(z[2], 100.0, o.p.dt) - 1) < 1e-7
    # u_z of (m,k)=(1,0) ~ J1(j11 r): rate j11^2/Re
    u = np.zeros((3, nr, 3, 2), complex)
    u[2, :, 2, 0] = 1e-8 * sp.jv(1, z[1] * o.r)
    u[2, :, 0, 0] = np.conj(u[2, :, 2, 0])
    assert abs(_decay_rate(o, u, 40) / _cn_rate(z[1], 100.0, o.p.dt) - 1) < 1e-7


# ---------------------------------------------------------------- step invariants
def test_step_keeps_wall_flux_and_hermitian_plane():
    o = _oracle()
    u = _field(o, 1, 1e-2)
    u1 = o.step(u, 0.3)
    assert np.abs(u1[:, 0]).max() < 1e-15
    assert abs(np.dot(o.W, u1[2, :, o.p.M, 0])) < 1e-16
    np.testing.assert_allclose(u1[:, :, ::-1, 0], np.conj(u1[:, :, :, 0]), atol=1e-17)
    assert np.all(u1[0, :, o.p.M, 0] == 0)


def test_divergence_converges_under_refinement():
    rel = []
    for nr in (16, 32, 48):
        o = _oracle(nr=nr, Re=100.0)
        u1 = o.step(_field(o, 1, 1e-2), 0.0)
        w = o.curl(u1)
        d = o.divergence(u1)
        rel.append(math.sqrt(np.sum(o.What * np.abs(d) ** 2) / o.inner(w, w)))
    assert rel[1] < rel[0] / 50 and rel[2] < rel[1] / 10 and rel[2] < 5e-6


def test_energy_budget_production_minus_dissipation():
    res = []
    for dt in (0.004, 0.002):
        # nr = 32: the spatial floor of the discrete budget (~1e-6) stays below the O(dt^2) time error
        o = _oracle(nr=32, M=2, K=2, Re=100.0, dt=dt)
        ns = int(round(0.2 / dt))
        u = o.forward(_field(o, 2, 1e-3), 0.0, ns)
        t = ns * dt
        u1 = o.step(u, t)
        u2 = o.step(u1, t + dt)
        dEdt = (o.energy(u2) - o.energy(u)) / (2 * dt)
        _, dU = o.base(t + dt)
        prod = -o.inner(u1[0], dU[:, None, None] * u1[2])
        w = o.curl(u1)
        diss = o.inner(w, w) / o.p.Re
        assert abs(prod) > 1e-3 * diss
        res.append(abs(dEdt - (prod - diss)) / diss)
    assert res[1] < 1e-5 and res[0] / res[1] > 3.0


def test_reflection_symmetry_theta_to_minus_theta():
    o = _oracle()
    u = _field(o, 8, 1e-2)

    def refl(f):
        g = f[:, :, ::-1, :].copy()
        g[1] *= -1
        return g

    np.testing.assert_allclose(o.step(refl(u), 0.2), refl(o.step(u, 0.2)), atol=1e-14 * np.abs(u).max())


def test_linear_mode_step_is_the_step_restricted_to_one_mode():
    o = _oracle(nr=12, M=3, K=4)
    for (m, k) in ((2, 3), (-3, 1), (1, 0), (0, 0)):
        um = synth.single_mode(o.r, m, k, o.p.Lz, seed=7) * 1e-12
        full = np.zeros((3, o.p.nr, 2 * o.p.M + 1, o.p.K + 1), np.complex128)
        full[:, :, m + o.p.M, k] = um
        if k == 0:
            full[:, :, -m + o.p.M, k] = np.conj(um)
        ref = o.step(full, 0.7)[:, :, m + o.p.M, k]
        got = o.linear_mode_step(um, m, k, 0.7)
        np.testing.assert_allclose(got, ref, atol=1e-9 * np.abs(ref).max())


# ---------------------------------------------------------------- adjoint
def _jvp(o, u, v, t, h=1.0):
    f = lambda e: o.step(u + e * v, t)
    return (f(-2 * h) - 8 * f(-h) + 8 * f(h) - f(2 * h)) / (12 * h)  # exact for quartic maps


def test_adjoint_step_dot_product():
    o = _oracle()
    u = _field(o, 1, 1e-2)
    v = _field(o, 5, 1e-2)
    w = synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=6)
    lhs = np.sum(np.real(np.conj(_jvp(o, u, v, 0.1)) * w))
    rhs = np.sum(np.real(np.conj(v) * o.adjoint_step(u, 0.1, w)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_step_equals_bruteforce_jacobian_transpose():
    o = _oracle(nr=8, M=1, K=1)
    u = _field(o, 2, 1e-1)
    shape = u.shape
    n = u.size
    J = np.zeros((2 * n, 2 * n))
    for c in range(2 * n):
        e = np.zeros(2 * n)
        e[c] = 1.0
        v = (e[:n] + 1j * e[n:]).reshape(shape)
        jv = _jvp(o, u, v, 0.0, h=1e-2).ravel()
        J[:, c] = np.r_[jv.real, jv.imag]
    rng = np.random.default_rng(0)
    for _ in range(3):
        wv = rng.standard_normal(2 * n)
        w = (wv[:n] + 1j * wv[n:]).reshape(shape)
        got = o.adjoint_step(u, 0.0, w).ravel()
        ref = J.T @ wv
        np.testing.assert_allclose(np.r_[got.real, got.imag], ref, atol=1e-9 * np.abs(ref).max())


@pytest.mark.slow
def test_gradient_matches_central_differences():
    o = _oracle(nr=12, M=2, K=2, dt=0.01)
    u0 = _field(o, 1, 1e-2)
    nsteps = 15
    ET, g = o.gradient(u0, 0.0, nsteps)
    for seed in (11, 12, 13):
        v = _field(o, seed, 1e-2)
        E = lambda e: o.energy(o.forward(u0 + e * v, 0.0, nsteps))
        D = lambda h: (E(h) - E(-h)) / (2 * h)
        h = 1e-2
        fd = (4 * D(h / 2) - D(h)) / 3
        assert abs(o.inner(g, v) - fd) <= 1e-6 * abs(fd)


# ---------------------------------------------------------------- checkpointing counts
def test_revolve_formula_equals_bruteforce_minimum():
    C = po.revolve_advances_dp(96, 6)
    for n in range(1, 97):
        for s in range(1, 7):
            assert C[n, s] == po.revolve_advances(n, s), (n, s)


def test_revolve_formula_closed_cases():
    assert po.revolve_advances(10, 1) == 45            # l(l-1)/2 with one slot
    for n in (5, 17, 200):
        assert po.revolve_advances(n, n) == n - 1      # store-all: one advance per step
    assert po.revolve_repetitions(4000, 32) == 3


# ---------------------------------------------------------------- planted mistakes
def test_planted_sign_error_in_base_term_breaks_energy_budget(monkeypatch):
    orig = po.Oracle.nonlinear

    def bad(self, u, t):
        n = orig(self, u, t)
        _, dU = self.base(t)
        n[2] += 2 * dU[:, None, None] * u[0]   # flips the sign of -dU/dr u_r
        return n

    monkeypatch.setattr(po.Oracle, "nonlinear", bad)
    with pytest.raises(AssertionError):
        test_energy_budget_production_minus_dissipation()


def test_planted_dropped_term_in_curl_transpose_breaks_dot_product(monkeypatch):
    orig = po.Oracle.curlT

    def bad(self, wb):
        out = orig(self, wb)
        out[1] -= wb[2] / self.r[:, None, None]   # drops the u_theta / r term
        return out

    monkeypatch.setattr(po.Oracle, "curlT", bad)
    with pytest.raises(AssertionError):
        test_adjoint_step_dot_product()


def test_planted_missing_hermitian_factor_breaks_library_transform(monkeypatch):
    def bad_synth(self, fh):
        x = np.einsum('am,jmk->jak', self.Et, fh)
        return np.real(np.einsum('jak,bk->jab', x, self.Ez))

    monkeypatch.setattr(po.Oracle, "synth", bad_synth)
    with pytest.raises(AssertionError):
        test_synth_matches_library_irfft()


def test_mode_energy_and_resolution_measures_follow_their_definitions():
    """Per-mode energies sum to the energy; e_M, e_K from the stored half
    spectrum equal the paper's sums over the full spectrum (Section 2.4),
    evaluated here from the Hermitian extension f(-m, -k) = conj f(m, k)."""
    from paper_2509_10103_gb300 import diagnostics, synth
    p = po.Params(nr=10, M=3, K=4, Lz=7.0, Re=1000.0, dt=0.01)
    o = po.Oracle(p)
    u = synth.random_field(o.r, p.M, p.K, p.Lz, seed=5, decay=1.5)
    spec = o.mode_energy(u)
    E = o.energy(u)
    assert abs(spec.sum() / E - 1) < 1e-13
    # full spectrum over k = -K..K
    W = 0.5 * (2 * math.pi * p.Lz) * o.W
    def e_full(m, k):
        f = u[:, :, m + p.M, k] if k >= 0 else np.conj(u[:, :, -m + p.M, -k])
        return float(np.sum(W * np.sum(np.abs(f) ** 2, axis=0)))
    total = sum(e_full(m, k) for m in range(-p.M, p.M + 1) for k in range(-p.K, p.K + 1))
    assert abs(total / E - 1) < 1e-12
    eM = sum(e_full(p.M, k) for k in range(-p.K, p.K + 1)) / E
    eK = sum(e_full(m, p.K) for m in range(-p.M, p.M + 1)) / E
    gM, gK = diagnostics.resolution_measures(spec, E)
    assert abs(gM / eM - 1) < 1e-12 and abs(gK / eK - 1) < 1e-12
    Grt, Gz = diagnostics.component_gains(spec, E)
    assert abs(Grt + Gz - 1) < 1e-13
    assert abs(Gz - float(np.sum(0.5 * o.What * np.abs(u[2]) ** 2)) / E) < 1e-13


def test_oracle_resolution_measures_on_fields_with_known_shells():
    """Oracle.resolution against facts fixed by the definitions: the full
    spectrum holds the whole energy; a field living only in the mode (M, k0)
    shares it equally with the conjugate partner (-M, -k0), so e_M = 1/2 and
    e_K = 0 for k0 < K; one only in (m0, K) has e_K = 1/2 likewise; removing
    those shells gives zero; and the values match the brute-force sums over
    the Hermitian extension."""
    from paper_2509_10103_gb300 import synth
    p = po.Params(nr=10, M=3, K=4, Lz=7.0, Re=1000.0, dt=0.01)
    o = po.Oracle(p)
    u = synth.random_field(o.r, p.M, p.K, p.Lz, seed=8, decay=1.5)
    E = o.energy(u)
    f = o.full_spectrum(u)
    assert f.shape == (3, p.nr, 2 * p.M + 1, 2 * p.K + 1)
    W = 0.5 * (2 * math.pi * p.Lz) * o.W
    assert abs(np.einsum('j,cjmk->', W, np.abs(f) ** 2) / E - 1) < 1e-13
    eM, eK = o.resolution(u, E)
    bM = sum(float(np.sum(W * np.sum(np.abs(u[:, :, p.M + p.M, k] if k >= 0 else np.conj(u[:, :, 0, -k])) ** 2,
                                         axis=0))) for k in range(-p.K, p.K + 1)) / E
    assert abs(eM / bM - 1) < 1e-12
    from paper_2509_10103_gb300 import diagnostics
    assert abs(eK / diagnostics.resolution_measures(o.mode_energy(u), E)[1] - 1) < 1e-12
    only = np.zeros_like(u)
    only[:, :, 2 * p.M, 2] = u[:, :, 2 * p.M, 2]
    assert o.resolution(only, o.energy(only)) == pytest.approx((0.5, 0.0), abs=1e-14)
    only = np.zeros_like(u)
    only[:, :, 1, p.K] = u[:, :, 1, p.K]
    assert o.resolution(only, o.energy(only)) == pytest.approx((0.0, 0.5), abs=1e-14)
    cut = u.copy()
    cut[:, :, 0, :] = 0
    cut[:, :, 2 * p.M, :] = 0
    cut[:, :, :, p.K] = 0
    assert o.resolution(cut, E) == (0.0, 0.0)


def test_linear_step_of_steady_pipe_flow_has_no_growing_mode():
    """Hagen-Poiseuille flow is linearly stable: the per-mode step map at
    Re = 1750 has every eigenvalue inside the unit circle (the rotational form
    of the base-flow terms fails this: a pair near 1.0016 at nr = 38)."""
    o = _oracle(nr=24, M=2, K=1, Lz=math.pi, Re=1750.0, dt=0.01, A=0.0)
    n = 3 * o.p.nr
    for m in range(0, 3):
        for k in range(0, 2):
            J = np.zeros((n, n), complex)
            for i in range(n):
                e = np.zeros(n, complex)
                e[i] = 1.0
                J[:, i] = o.linear_mode_step(e.reshape(3, o.p.nr), m, k, 0.0).ravel()
            assert np.abs(np.linalg.eigvals(J)).max() < 1.0, (m, k)


def test_uniform_base_flow_only_translates_a_mode():
    """The advective base-flow term -U du/dz (Eq. 2.5) for a plug flow U = U0:
    advection by a uniform velocity is a translation, so every Fourier mode of
    the solution without base flow turns by exp(-i k_z U0 t) (the factor is a
    scalar per mode and commutes with the viscous operator and the wall
    conditions).  The discrete pressure projection sees the forcing -i k_z U0 u
    through its discrete divergence, which vanishes only to finite-difference
    order, so the gap is a spatial discretisation error: it falls under radial
    refinement.  A wrong sign or a dropped k_z leaves an O(1) gap.  (The
    energy budget does not see this term: it is energy-neutral.)"""
    U0, T, m, k, dt = 0.7, 1.0, 1, 2, 0.01
    gaps = {}
    for nr in (12, 24):
        prm = dict(nr=nr, M=2, K=3, Lz=6.0, Re=1000.0, dt=dt, Wo=8.0, A=0.0, base=False)
        still = po.Oracle(po.Params(**prm))
        plug = po.Oracle(po.Params(**prm))
        plug.base = lambda t, o=plug: (np.full_like(o.r, U0), np.zeros_like(o.r))
        u = synth.random_field(still.r, 2, 3, 6.0, seed=9)[:, :, m + 2, k]
        a, b = u.copy(), u.copy()
        for s in range(int(round(T / dt))):
            a = still.linear_mode_step(a, m, k, s * dt)
            b = plug.linear_mode_step(b, m, k, s * dt)
        turn = np.exp(-1j * still.kz[k] * U0 * T)
        gaps[nr] = np.abs(b - a * turn).max() / np.abs(a).max()
        assert np.abs(b - a * np.conj(turn)).max() / np.abs(a).max() > 0.5  # the other direction is far off
    assert gaps[24] < 1e-4 and gaps[12] > 10 * gaps[24]


def paper_numbers():
    """Key -> value of tests/golden/paper_appendix_a.txt (numbers the paper prints)."""
    out = {}
    with open(os.path.join(GOLDEN, "paper_appendix_a.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()[:2]
                out[key] = float(val)
    return out


def test_printed_wo2_peak_fixes_the_time_unit():
    """App. A.2 prints the Wo = 2 growth peak both as t ~ 90 and as 0.029 T.
    With lengths in R and velocities in 2 U_bar the period is 2 pi Re / Wo^2
    (= 3141.6 at Re = 2000, Wo = 2) and 0.029 T = 91; the formula printed in
    the paper's introduction, pi Re / (2 Wo^2), would put the peak at 23.  The
    library and the oracle take the first (design reading 1)."""
    P = paper_numbers()
    Re, Wo = 2000.0, 2.0
    T_units = 2 * math.pi * Re / Wo ** 2
    T_printed = math.pi * Re / (2 * Wo ** 2)
    assert abs(P["wo2_re2000_a1_lz10_tpeak_over_T"] * T_units - P["wo2_re2000_a1_lz10_tpeak"]) < 2.0
    assert abs(P["wo2_re2000_a1_lz10_tpeak_over_T"] * T_printed - P["wo2_re2000_a1_lz10_tpeak"]) > 50.0
    o = po.Oracle(po.Params(nr=9, M=1, K=1, Lz=4.0, Re=Re, dt=0.01, Wo=Wo, A=1.0))
    # the oracle's base flow repeats after T_units: the bulk velocity u_b(t) = (1 + A sin(2 pi t / T)) / 2
    U0, _ = o.base(0.3)
    U1, _ = o.base(0.3 + T_units)
    Uh, _ = o.base(0.3 + 0.5 * T_units)
    assert np.abs(U1 - U0).max() < 1e-12 and np.abs(Uh - U0).max() > 1e-2  # T is the period, not a multiple
