"""Plain FP64 CPU oracle of the forward and adjoint pipe-flow time step.

TEST INFRASTRUCTURE ONLY.  This module is imported by the test-suite, by the
package-level smoke check and by the CPU-baseline leg of the benchmark; the
product path never imports it, and it shares no code with the CUDA library.

It restates, slowly and with dense per-mode matrices, the discrete scheme that
the CUDA path implements (Keuchel & Avila, "Nonlinear optimal perturbation
growth in pulsatile pipe flow"):

* perturbation Navier-Stokes about the Sexl-Womersley base flow, Eq. (2.5)-(2.7)
  with the pressure split p' = f_z z + p_hat of Section 2 (zero-bulk
  constraint, Eq. 2.7), in rotational form;
* Fourier-Galerkin in theta and z, Eq. (2.16), 3/2-rule dealiasing; high-order
  finite differences on Chebyshev radial points, Section 2.4;
* second-order predictor-corrector in time with the wall conditions imposed by
  an influence-matrix correction and the flux forcing f_z adjusted in each
  stage, Section 2.4;
* the discrete adjoint (exact transpose of the step) that replaces the
  continuous adjoint Eq. (2.9)-(2.11); the terminal condition is the
  compatibility condition Eq. (2.8) and the result is the gradient of
  Eq. (2.12) without the lambda term;
* the energy and inner product of Eq. (2.1)-(2.2).

Where the paper leaves the discretisation open the choices below are the ones
the library documents (radial grid, 9-point stencils with parity-mirrored axis
points, c = 1/2 Crank-Nicolson viscous part, one predictor and one corrector,
the influence correction on the pressure's wall datum, quadrature exact for
polynomials in r^2).  Layout of a field: complex128 [3][Nr][2M+1][K+1],
components (r, theta, z), j = 0 at the wall, m = -M..M, k = 0..K.

The adjoint step works with Euclidean cotangents of the stored real and
imaginary parts (reverse-mode differentiation of the discrete step); the
gradient returned by `gradient` is the Riesz representer in the energy inner
product, i.e. the Euclidean gradient divided by the quadrature weights.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

STENCIL = 9  # points per finite-difference stencil (Section 2.4: high order in r)


# --------------------------------------------------------------------------
# Radial grid, quadrature and finite differences (Section 2.4)
# --------------------------------------------------------------------------

def radial_grid(nr: int, stretch: float = 0.0) -> np.ndarray:
    """Chebyshev points of Section 2.4: the positive half of the 2Nr-point
    Chebyshev-Lobatto set, r_j = cos(pi j / (2Nr - 1)), blended with the uniform
    grid of the same end points by `stretch` (the paper's unstated relaxation)."""
    j = np.arange(nr, dtype=np.float64)
    x = np.cos(np.pi * j / (2 * nr - 1))
    rho = 1.0 - j * (1.0 - x[-1]) / (nr - 1)
    return (1.0 - stretch) * x + stretch * rho


def radial_weights(r: np.ndarray) -> np.ndarray:
    """Weights W_j with sum_j W_j f(r_j) = int_0^1 f(r) r dr (radial part of Eq. 2.2).

    With s = r^2 the integral is (1/2) int_0^1 f ds; W_j is half the integral of the
    j-th Lagrange basis polynomial in s over [0, 1], evaluated by Gauss-Legendre
    quadrature with as many nodes as grid points (exact for that degree)."""
    s = r ** 2
    n = len(r)
    xg, wg = np.polynomial.legendre.leggauss(n)
    sg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg
    w = np.zeros(n)
    for j in range(n):
        lj = np.ones_like(sg)
        for i in range(n):
            if i != j:
                lj *= (sg - s[i]) / (s[j] - s[i])
        w[j] = 0.5 * np.dot(lj, wg)
    return w


def fornberg(x0: float, x: np.ndarray, nd: int) -> np.ndarray:
    """Finite-difference weights c[i, d] for derivative d <= nd at x0 on nodes x
    (Fornberg 1988, 'Generation of finite difference formulas on arbitrarily
    spaced grids')."""
    n = len(x)
    c = np.zeros((n, nd + 1))
    c1 = 1.0
    c4 = x[0] - x0
    c[0, 0] = 1.0
    for i in range(1, n):
        mn = min(i, nd)
        c2 = 1.0
        c5 = c4
        c4 = x[i] - x0
        for j in range(i):
            c3 = x[i] - x[j]
            c2 *= c3
            if j == i - 1:
                for d in range(mn, 0, -1):
                    c[i, d] = c1 * (d * c[i - 1, d - 1] - c5 * c[i - 1, d]) / c2
                c[i, 0] = -c1 * c5 * c[i - 1, 0] / c2
            for d in range(mn, 0, -1):
                c[j, d] = (c4 * c[j, d] - d * c[j, d - 1]) / c3
            c[j, 0] = c4 * c[j, 0] / c3
        c1 = c2
    return c


def fd_matrices(r: np.ndarray, parity: int):
    """Dense D1, D2 (Nr x Nr) for a field of the given axis parity.

    Row j uses the 9 nearest points of the mirrored grid {r} U {-r} (one-sided at the
    wall).  A mirrored point -r_i carries the value parity * f(r_i)."""
    nr = len(r)
    ext = np.concatenate([r, -r[::-1]])
    d1 = np.zeros((nr, nr))
    d2 = np.zeros((nr, nr))
    for j in range(nr):
        lo = min(max(j - STENCIL // 2, 0), 2 * nr - STENCIL)
        idx = np.arange(lo, lo + STENCIL)
        c = fornberg(r[j], ext[idx], 2)
        for t, e in enumerate(idx):
            if e < nr:
                col, sg = e, 1.0
            else:
                col, sg = 2 * nr - 1 - e, float(parity)
            d1[j, col] += sg * c[t, 1]
            d2[j, col] += sg * c[t, 2]
    return d1, d2


# --------------------------------------------------------------------------
# Sexl-Womersley base flow (Eq. 2.3-2.4 and the Section 2 text)
# --------------------------------------------------------------------------

def bessel_j(nu: int, z) -> np.ndarray:
    """J_nu(z) for complex z by its power series (textbook definition)."""
    z = np.asarray(z, dtype=np.complex128)
    half = z / 2.0
    term = half ** nu / math.factorial(nu)
    total = term.copy()
    q = -(half * half)
    for k in range(1, 200):
        term = term * q / (k * (k + nu))
        total = total + term
        if np.all(np.abs(term) <= 1e-18 * np.maximum(np.abs(total), 1e-300)):
            break
    return total


def womersley(r: np.ndarray, t: float, Re: float, Wo: float, A: float):
    """U(r,t) and dU/dr in units of radius and 2 x mean bulk velocity.

    Steady part 1 - r^2 (Eq. 2.3) plus the oscillatory Stokes-layer solution whose
    bulk velocity 2 int U r dr equals u_b(t) = (1 + A sin(w t)) / 2 (Eq. 2.4), with
    w = Wo^2 / Re (period 2 pi Re / Wo^2 in these units) and kappa = i^(3/2) Wo."""
    r = np.asarray(r, dtype=np.float64)
    U = 1.0 - r * r
    dU = -2.0 * r
    if A == 0.0:
        return U, dU
    omega = Wo * Wo / Re
    kappa = np.exp(0.75j * np.pi) * Wo
    j0k = bessel_j(0, kappa)
    j1k = bessel_j(1, kappa)
    B = (-0.5j * A) / (1.0 - 2.0 * j1k / (kappa * j0k))
    prof = B * (1.0 - bessel_j(0, kappa * r) / j0k)
    dprof = B * kappa * bessel_j(1, kappa * r) / j0k
    ph = np.exp(1j * omega * t)
    return U + np.real(prof * ph), dU + np.real(dprof * ph)


# --------------------------------------------------------------------------
# Problem set-up
# --------------------------------------------------------------------------

@dataclass
class Params:
    nr: int
    M: int
    K: int
    Lz: float
    Re: float
    dt: float
    Wo: float = 8.0
    A: float = 1.0
    stretch: float = 0.0
    base: bool = True  # False: no base flow (U = 0), used by the Stokes-decay pins


@dataclass
class Oracle:
    p: Params
    r: np.ndarray = field(init=False)
    W: np.ndarray = field(init=False)

    def __post_init__(self):
        p = self.p
        self.r = radial_grid(p.nr, p.stretch)
        self.W = radial_weights(self.r)
        self.m = np.arange(-p.M, p.M + 1)
        self.kz = 2.0 * np.pi * np.arange(p.K + 1) / p.Lz
        self.ck = np.where(np.arange(p.K + 1) == 0, 1.0, 2.0)
        self.D = {+1: fd_matrices(self.r, +1), -1: fd_matrices(self.r, -1)}
        self.ntheta = 3 * (p.M + 1)
        self.nz = 3 * (p.K + 1)
        # exact DFT matrices of the 3/2-padded grid; negative m are conjugates of positive m
        a = np.arange(self.ntheta)
        et = np.zeros((self.ntheta, 2 * p.M + 1), np.complex128)
        for m in range(0, p.M + 1):
            col = np.exp(2j * np.pi * ((m * a) % self.ntheta) / self.ntheta)
            et[:, p.M + m] = col
            et[:, p.M - m] = np.conj(col)
        b = np.arange(self.nz)
        ez = np.zeros((self.nz, p.K + 1), np.complex128)
        for k in range(p.K + 1):
            ez[:, k] = np.exp(2j * np.pi * ((k * b) % self.nz) / self.nz)
        self.Et, self.Ez = et, ez
        # energy weights W_hat[j, k] = 2 pi Lz W_j c_k  (Eq. 2.2 with Hermitian doubling)
        self.What = (2.0 * np.pi * p.Lz) * self.W[:, None, None] * self.ck[None, None, :]
        self._maps = {}

    # ---------------- inner products (Eq. 2.1-2.2) ----------------
    def inner(self, a: np.ndarray, b: np.ndarray) -> float:
        return float(np.sum(self.What[None] * np.real(np.conj(a) * b)))

    def energy(self, u: np.ndarray) -> float:
        return 0.5 * self.inner(u, u)

    # ---------------- radial operators ----------------
    def par(self, m: int) -> int:
        return 1 if m % 2 == 0 else -1

    def d1(self, m_par: int):
        return self.D[self.par(m_par)][0]

    def lap(self, mm: int, kz: float) -> np.ndarray:
        d1, d2 = self.D[self.par(mm)]
        r = self.r
        return d2 + d1 / r[:, None] - np.diag(mm * mm / r ** 2 + kz * kz)

    def apply_d1(self, f: np.ndarray, shift: int) -> np.ndarray:
        """D1 along r for every mode of f[Nr, 2M+1, K+1]; parity (-1)^(m+shift)."""
        out = np.empty_like(f)
        for i, m in enumerate(self.m):
            out[:, i, :] = self.d1(m + shift) @ f[:, i, :]
        return out

    def apply_d1T(self, f: np.ndarray, shift: int) -> np.ndarray:
        out = np.empty_like(f)
        for i, m in enumerate(self.m):
            out[:, i, :] = self.d1(m + shift).T @ f[:, i, :]
        return out

    # ---------------- curl (spectral, mode by mode) ----------------
    def curl(self, u: np.ndarray) -> np.ndarray:
        ur, ut, uz = u
        imr = 1j * self.m[None, :, None] / self.r[:, None, None]
        ikz = 1j * self.kz[None, None, :]
        wr = imr * uz - ikz * ut
        wt = ikz * ur - self.apply_d1(uz, 0)
        wz = self.apply_d1(ut, 1) + ut / self.r[:, None, None] - imr * ur
        return np.stack([wr, wt, wz])

    def curlT(self, wb: np.ndarray) -> np.ndarray:
        wr, wt, wz = wb
        imr = 1j * self.m[None, :, None] / self.r[:, None, None]
        ikz = 1j * self.kz[None, None, :]
        ur = -ikz * wt + imr * wz
        ut = ikz * wr + self.apply_d1T(wz, 1) + wz / self.r[:, None, None]
        uz = -imr * wr - self.apply_d1T(wt, 0)
        return np.stack([ur, ut, uz])

    # ---------------- 3/2-padded transforms (Eq. 2.16) ----------------
    def synth(self, fh: np.ndarray) -> np.ndarray:
        """f(theta_a, z_b) = sum_k c_k Re(sum_m fh[m,k] e^{i m theta_a} e^{i kz z_b})."""
        x = np.einsum('am,jmk->jak', self.Et, fh * self.ck[None, None, :])
        return np.real(np.einsum('jak,bk->jab', x, self.Ez))

    def _herm(self, fh: np.ndarray) -> np.ndarray:
        M = self.p.M
        out = fh.copy()
        k0 = fh[:, :, 0]
        out[:, :, 0] = 0.5 * (k0 + np.conj(k0[:, ::-1]))
        return out

    def analysis(self, g: np.ndarray) -> np.ndarray:
        """Truncated DFT / (N_theta N_z) onto |m| <= M, 0 <= k <= K, Hermitian at k = 0."""
        x = np.einsum('am,jab->jmb', np.conj(self.Et), g)
        fh = np.einsum('jmb,bk->jmk', x, np.conj(self.Ez)) / (self.ntheta * self.nz)
        return self._herm(fh)

    def analysisT(self, hb: np.ndarray) -> np.ndarray:
        """Transpose of `analysis` for Euclidean cotangents."""
        return self.synth(hb / self.ck[None, None, :]) / (self.ntheta * self.nz)

    def synthT(self, gb: np.ndarray) -> np.ndarray:
        """Transpose of `synth` for Euclidean cotangents: c_k sum g e^{-i phi}."""
        x = np.einsum('am,jab->jmb', np.conj(self.Et), gb)
        fh = np.einsum('jmb,bk->jmk', x, np.conj(self.Ez)) * self.ck[None, None, :]
        return self._herm(fh)

    # ---------------- nonlinear forcing (Eq. 2.5: quadratic term rotational, base-flow terms advective) ----------------
    def base(self, t: float):
        p = self.p
        if not p.base:
            z = np.zeros_like(self.r)
            return z, z
        return womersley(self.r, t, p.Re, p.Wo, p.A)

    def nonlinear(self, u: np.ndarray, t: float) -> np.ndarray:
        """N = u x w - U du/dz - u_r dU/dr e_z, w = curl u: the quadratic term in
        rotational form, the base-flow terms in advective form (they differ from
        (U e_z) x w + u x (-dU/dr e_theta) by grad(U u_z), which the discrete
        projection does not remove exactly)."""
        w = self.curl(u)
        up = np.stack([self.synth(c) for c in u])
        wp = np.stack([self.synth(c) for c in w])
        cr = np.cross(up, wp, axis=0)
        n = np.stack([self.analysis(c) for c in cr])
        U, dU = self.base(t)
        a = -1j * self.kz[None, None, :] * U[:, None, None]  # -U d/dz
        n += a[None] * u
        n[2] += -dU[:, None, None] * u[0]
        return n

    def nonlinearT(self, u: np.ndarray, t: float, nb: np.ndarray) -> np.ndarray:
        """Transpose of the Jacobian of `nonlinear` at u applied to the cotangent nb."""
        w = self.curl(u)
        up = np.stack([self.synth(c) for c in u])
        wp = np.stack([self.synth(c) for c in w])
        gb = np.stack([self.analysisT(c) for c in nb])
        upb = np.cross(wp, gb, axis=0)
        wpb = np.cross(gb, up, axis=0)
        ub = np.stack([self.synthT(c) for c in upb])
        wb = np.stack([self.synthT(c) for c in wpb])
        U, dU = self.base(t)
        a = -1j * self.kz[None, None, :] * U[:, None, None]
        ub += np.conj(a)[None] * nb          # y = a x  ->  x_bar = conj(a) y_bar
        ub[0] += -dU[:, None, None] * nb[2]
        return ub + self.curlT(wb)

    # ---------------- linear stage map S(u, F) (Section 2.4) ----------------
    def mode_maps(self, m: int, k: int):
        """Dense (3Nr x 3Nr) matrices Su, SF with u_new = Su u + SF F for mode (m, k)."""
        key = (m, k)
        if key in self._maps:
            return self._maps[key]
        p = self.p
        nr = p.nr
        r = self.r
        kz = self.kz[k]
        I = np.eye(nr)
        Z = np.zeros((nr, nr))
        E = np.diag(np.r_[0.0, np.ones(nr - 1)])
        e0 = np.zeros(nr)
        e0[0] = 1.0
        d1p = self.d1(m)        # parity of p and u_z
        d1v = self.d1(m + 1)    # parity of u_r, u_theta
        is00 = (m == 0 and k == 0)
        # divergence (Nr x 3Nr) and gradient (3Nr x Nr)
        Dv = np.hstack([d1v + np.diag(1.0 / r), np.diag(1j * m / r), 1j * kz * I])
        G = np.vstack([d1p + 0j, np.diag(1j * m / r), 1j * kz * I])
        # pressure: L_m p = div F inside, dp/dr = 0 at the wall (tentative datum)
        Ap = self.lap(m, kz).astype(np.complex128)
        Ap[0, :] = d1p[0, :]
        if is00:
            Proj = np.eye(3 * nr, dtype=np.complex128)
        else:
            Proj = np.eye(3 * nr) - G @ np.linalg.solve(Ap, E @ Dv)
        # +/- basis: u+ = u_r + i u_t, u- = u_r - i u_t
        T = np.block([[I, 1j * I, Z], [I, -1j * I, Z], [Z, Z, I]])
        Ti = np.block([[0.5 * I, 0.5 * I, Z], [-0.5j * I, 0.5j * I, Z], [Z, Z, I]])
        Hu = np.zeros((3 * nr, 3 * nr), np.complex128)
        HF = np.zeros((3 * nr, 3 * nr), np.complex128)
        for blk, mm in enumerate((m + 1, m - 1, m)):
            L = self.lap(mm, kz)
            Av = I / p.dt - L / (2.0 * p.Re)
            Av[0, :] = e0
            Bv = I / p.dt + L / (2.0 * p.Re)
            s = slice(blk * nr, (blk + 1) * nr)
            Hu[s, s] = np.linalg.solve(Av, E @ Bv)
            HF[s, s] = np.linalg.solve(Av, E)
        Su = Ti @ Hu @ T
        SF = Ti @ HF @ T @ Proj
        if is00:
            # flux forcing f_z (Eq. 2.7): u_z += f g with int u_z r dr = 0; u_r = 0
            L0 = self.lap(0, 0.0)
            A0 = I / p.dt - L0 / (2.0 * p.Re)
            A0[0, :] = e0
            g = np.linalg.solve(A0, E @ np.ones(nr))
            Fin = np.eye(3 * nr, dtype=np.complex128)
            Fin[2 * nr:, 2 * nr:] += np.outer(g, -self.W / np.dot(self.W, g))
            Fin[:nr, :] = 0.0
        else:
            # influence correction of the pressure's wall datum: the response h to a
            # unit Neumann datum is added so that div u = 0 at the wall
            phi = np.linalg.solve(Ap, e0.astype(np.complex128))
            h = Ti @ HF @ T @ (-(G @ phi))
            delta = d1v[0, :] @ h[:nr]
            crow = np.zeros(3 * nr, np.complex128)
            crow[:nr] = -d1v[0, :] / delta
            Fin = np.eye(3 * nr, dtype=np.complex128) + np.outer(h, crow)
        out = (Fin @ Su, Fin @ SF)
        self._maps[key] = out
        return out

    def _apply(self, u: np.ndarray, F: np.ndarray | None, transpose: bool):
        nr = self.p.nr
        out_u = np.zeros_like(u)
        out_F = np.zeros_like(u)
        for i, m in enumerate(self.m):
            for k in range(self.p.K + 1):
                Su, SF = self.mode_maps(int(m), k)
                uv = u[:, :, i, k].reshape(3 * nr)
                if not transpose:
                    res = Su @ uv + SF @ F[:, :, i, k].reshape(3 * nr)
                    out_u[:, :, i, k] = res.reshape(3, nr)
                else:
                    out_u[:, :, i, k] = (Su.conj().T @ uv).reshape(3, nr)
                    out_F[:, :, i, k] = (SF.conj().T @ uv).reshape(3, nr)
        return out_u, out_F

    def stage(self, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        return self._apply(u, F, False)[0]

    def stageT(self, ub: np.ndarray):
        """Cotangents (of u, of F) from the cotangent of the stage output."""
        return self._apply(ub, None, True)

    # ---------------- time step (predictor-corrector, Section 2.4) ----------------
    def step(self, u: np.ndarray, t: float) -> np.ndarray:
        n0 = self.nonlinear(u, t)
        us = self.stage(u, n0)
        n1 = self.nonlinear(us, t + self.p.dt)
        return self.stage(u, 0.5 * (n0 + n1))

    def step_stages(self, u: np.ndarray, t: float):
        n0 = self.nonlinear(u, t)
        us = self.stage(u, n0)
        n1 = self.nonlinear(us, t + self.p.dt)
        return n0, us, n1, self.stage(u, 0.5 * (n0 + n1))

    def adjoint_step(self, u: np.ndarray, t: float, lb: np.ndarray) -> np.ndarray:
        """Euclidean cotangent of u^n from that of u^{n+1}; re-runs the predictor."""
        n0 = self.nonlinear(u, t)
        us = self.stage(u, n0)
        ub, Fb = self.stageT(lb)
        usb = self.nonlinearT(us, t + self.p.dt, 0.5 * Fb)
        ub2, n0b = self.stageT(usb)
        ub = ub + ub2
        n0b = n0b + 0.5 * Fb
        return ub + self.nonlinearT(u, t, n0b)

    def forward(self, u0: np.ndarray, t0: float, nsteps: int, keep: bool = False):
        u = u0.copy()
        states = [u.copy()] if keep else None
        for n in range(nsteps):
            u = self.step(u, t0 + n * self.p.dt)
            if keep:
                states.append(u.copy())
        return (u, states) if keep else u

    def gradient(self, u0: np.ndarray, t0: float, nsteps: int):
        """E(T) and the Riesz gradient dE(T)/du0 (store-all reverse sweep).

        Terminal cotangent W_hat u_N is the compatibility condition Eq. (2.8) with the
        sign of the paper's u_dagger reversed (u_dagger = -gradient)."""
        uN, states = self.forward(u0, t0, nsteps, keep=True)
        ET = self.energy(uN)
        lb = self.What[None] * uN
        for n in range(nsteps - 1, -1, -1):
            lb = self.adjoint_step(states[n], t0 + n * self.p.dt, lb)
        return ET, lb / self.What[None]

    def linear_mode_step(self, um: np.ndarray, m: int, k: int, t: float) -> np.ndarray:
        """`step` restricted to one Fourier mode (um: 3 x Nr) for a vanishing
        amplitude: the u x w term drops and the base-flow terms act mode by mode."""
        p = self.p

        def forcing(v, tt):
            U, dU = self.base(tt)
            a = -1j * self.kz[k] * U
            return np.stack([a * v[0], a * v[1], a * v[2] - dU * v[0]])

        Su, SF = self.mode_maps(m, k)
        n0 = forcing(um, t)
        us = (Su @ um.ravel() + SF @ n0.ravel()).reshape(3, p.nr)
        n1 = forcing(us, t + p.dt)
        return (Su @ um.ravel() + SF @ (0.5 * (n0 + n1)).ravel()).reshape(3, p.nr)

    # ---------------- diagnostics used by the pins ----------------
    def divergence(self, u: np.ndarray) -> np.ndarray:
        ur, ut, uz = u
        imr = 1j * self.m[None, :, None] / self.r[:, None, None]
        ikz = 1j * self.kz[None, None, :]
        return self.apply_d1(ur, 1) + ur / self.r[:, None, None] + imr * ut + ikz * uz

    # ---------------- continuous adjoint (Eq. 2.9-2.11), the paper's own form ----------------
    def grad_u(self, u: np.ndarray):
        """Velocity-gradient tensor G[i][j] = (grad u)_ij in cylindrical components
        (i the derivative direction r, theta, z; j the velocity component), spectral:
        (d_r u_j), ((d_theta u_r - u_theta)/r, (d_theta u_theta + u_r)/r, d_theta u_z / r),
        (d_z u_j)."""
        ur, ut, uz = u
        ir = 1.0 / self.r[:, None, None]
        im = 1j * self.m[None, :, None]
        ikz = 1j * self.kz[None, None, :]
        return [[self.apply_d1(ur, 1), self.apply_d1(ut, 1), self.apply_d1(uz, 0)],
                [(im * ur - ut) * ir, (im * ut + ur) * ir, im * uz * ir],
                [ikz * ur, ikz * ut, ikz * uz]]

    def nonlinear_adj(self, w: np.ndarray, u: np.ndarray, t: float) -> np.ndarray:
        """Forcing of the adjoint equation (Eq. 2.9) in backward time tau = T - t:
        dw/dtau = Re^-1 lap w + N_adj(w; u) - grad p_dagger, with
        N_adj = ((U + u).grad) w - (grad(U + u)) . w
              = U dw/dz - w_z dU/dr e_r  +  P[-u x curl w - 2 (grad u) . w],
        the gradient part grad(u . w) of the perturbation term going into the adjoint
        pressure, the base-flow part in advective form (as in `nonlinear`)."""
        om = self.curl(w)
        up = np.stack([self.synth(c) for c in u])
        wp = np.stack([self.synth(c) for c in w])
        omp = np.stack([self.synth(c) for c in om])
        G = self.grad_u(u)
        Gp = [[self.synth(G[i][j]) for j in range(3)] for i in range(3)]
        Gw = np.stack([sum(Gp[i][j] * wp[j] for j in range(3)) for i in range(3)])
        n = np.stack([self.analysis(c) for c in (-np.cross(up, omp, axis=0) - 2.0 * Gw)])
        U, dU = self.base(t)
        n += (1j * self.kz[None, None, :] * U[:, None, None])[None] * w
        n[0] += -dU[:, None, None] * w[2]
        return n

    def adjoint_step_continuous(self, u_next: np.ndarray, t_next: float, u_now: np.ndarray, t_now: float,
                                w: np.ndarray) -> np.ndarray:
        """w(t_now) from w(t_next), t_next = t_now + dt: the predictor-corrector of
        `step` run backward in time with the adjoint forcing, taken at (u_next,
        t_next) for the predictor and at (u_now, t_now) for the corrector."""
        n0 = self.nonlinear_adj(w, u_next, t_next)
        ws = self.stage(w, n0)
        n1 = self.nonlinear_adj(ws, u_now, t_now)
        return self.stage(w, 0.5 * (n0 + n1))

    def gradient_continuous(self, u0: np.ndarray, t0: float, nsteps: int):
        """E(T) and the gradient from the continuous adjoint: w(T) = u(T) (the
        compatibility condition Eq. 2.8 with w = -u_dagger), integrated back to t0;
        w(t0) is the gradient in the energy inner product (w = -u_dagger, Eq. 2.12)."""
        uN, states = self.forward(u0, t0, nsteps, keep=True)
        w = uN.copy()
        for n in range(nsteps - 1, -1, -1):
            w = self.adjoint_step_continuous(states[n + 1], t0 + (n + 1) * self.p.dt, states[n],
                                             t0 + n * self.p.dt, w)
        return self.energy(uN), w

    def mode_energy(self, u: np.ndarray) -> np.ndarray:
        """Energy of each stored mode (m, k >= 0) with the weights of Eq. 2.1, split
        into the cross-section part (u_r, u_theta) [0] and the axial part (u_z) [1];
        shape (2, 2M+1, K+1), summing to `energy`."""
        w = 0.5 * self.What
        a = np.sum(w * (np.abs(u[0]) ** 2 + np.abs(u[1]) ** 2), axis=0)
        b = np.sum(w * np.abs(u[2]) ** 2, axis=0)
        return np.stack([a, b])

    def full_spectrum(self, u: np.ndarray) -> np.ndarray:
        """Coefficients of every mode k = -K..K (axis 3, index k + K) from the
        stored half by the Hermitian symmetry f(-m, -k) = conj f(m, k) (Eq. 2.16)."""
        K = self.p.K
        neg = np.conj(u[:, :, ::-1, :0:-1])      # (m, -k) = conj(-m, k), k = K..1
        return np.concatenate([neg, u], axis=3)

    def resolution(self, u: np.ndarray, E0: float):
        """Resolution measures of Section 2.4: the energy in the highest
        azimuthal mode m = M summed over k = -K..K, and in the highest axial
        mode k = K summed over m = -M..M, each over E0.  (The printed formulas
        are garbled; they are read as energy fractions of these mode shells,
        with the energy of Eq. 2.1 and each mode of the full spectrum counted
        once.)"""
        p = self.p
        f = self.full_spectrum(u)
        w = 0.5 * (2.0 * np.pi * p.Lz) * self.W            # per radial point, one full-spectrum mode
        e = np.einsum('j,cjmk->mk', w, np.abs(f) ** 2)      # energy of every (m, k), k = -K..K
        return float(e[2 * p.M, :].sum() / E0), float(e[:, 2 * p.K].sum() / E0)

    def scale_to(self, u: np.ndarray, E0: float) -> np.ndarray:
        return u * math.sqrt(E0 / self.energy(u))


# --------------------------------------------------------------------------
# Binomial checkpointing counts (Section 2.5, Eq. 2.18-2.20)
# --------------------------------------------------------------------------

def beta(s: int, t: int) -> int:
    """beta(s, t) = C(s + t, s), Eq. (2.20)."""
    if t < 0:
        return 0
    return math.comb(s + t, s)


def revolve_repetitions(nsteps: int, snaps: int) -> int:
    """The unique r with beta(snaps, r-1) < nsteps <= beta(snaps, r), Eq. (2.19)."""
    r = 0
    while beta(snaps, r) < nsteps:
        r += 1
    return r


def revolve_advances(nsteps: int, snaps: int) -> int:
    """Minimal number of recomputed forward steps, Eq. (2.18):
    N_rec = S N - beta(N_G + 1, S - 1), S the repetition number of Eq. (2.19)."""
    if nsteps <= 1:
        return 0
    r = revolve_repetitions(nsteps, snaps)
    return r * nsteps - beta(snaps + 1, r - 1)


def revolve_advances_dp(nmax: int, smax: int) -> np.ndarray:
    """Brute-force minimum over all split points, C[l, s], for the taped-step model.

    Reversing l steps from a stored state with s snapshot slots (the stored start
    state included): either one step is reversed directly (l = 1), or with one
    slot every step i < l is recomputed from the start, or the range is split at
    m: advance m steps, store, reverse the tail with s - 1 slots, then the head."""
    INF = 1 << 60
    C = np.full((nmax + 1, smax + 1), INF, dtype=np.int64)
    for s in range(1, smax + 1):
        C[0, s] = 0
        C[1, s] = 0
    for l in range(2, nmax + 1):
        C[l, 1] = l * (l - 1) // 2
        for s in range(2, smax + 1):
            best = INF
            for m in range(1, l):
                v = m + C[l - m, s - 1] + C[m, s]
                if v < best:
                    best = v
            C[l, s] = best
    return C
