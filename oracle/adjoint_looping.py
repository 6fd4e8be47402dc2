"""Plain CPU oracle of the adjoint-looping optimisation (Section 2.3).

TEST INFRASTRUCTURE ONLY.  Imported by the test-suite; the product path never
imports it, and it shares no code with the CUDA library.

Gradient ascent on the energy shell E(u0) = E0 (Section 2.3, "Optimization
step"):

* update  u^{s+1} = (1 + lambda alpha) u^s - alpha u_dagger^s  (Eq. 2.13), with
  u_dagger = -grad E(T), the Riesz gradient of the final energy in the energy
  inner product (the paper's adjoint field at t = 0);
* lambda from the energy constraint E(u^{s+1}) = E0, the root lambda_+ of the
  quadratic (Eq. 2.14), with C0 = <u, u_dagger> and E0_dagger = <u_dagger, u_dagger>/2;
* real roots need 0 < alpha <= alpha_max (Eq. 2.15);
* backtracking: alpha = alpha_max first, halved while G does not grow, until G
  grows or R = |G^{s+1} - G^s| / G^{s+1} falls below the tolerance (10^-8 in
  the paper), which also ends the loop.

The paper's perturbations are admissible fields: solenoidal, zero at the wall
(no slip), with zero bulk flux (Section 2.2).  The gradient of the discrete
map with respect to all stored coefficients also has components outside that
set (reading: over all coefficients the optimum piles energy into the wall
row, where the quadrature weight is smallest).  The loop therefore works in
the admissible subspace V = {u(r=1) = 0, D u = 0 at every radial point, zero
flux and u_r = 0 for the mean mode, Hermitian k = 0 plane}, D the discrete
divergence of the scheme, with the gradient replaced by its orthogonal
projection onto V in the energy inner product (the gradient of E(T)
restricted to V).  A trial whose forward sweep is not finite counts as "G did
not grow".
"""
from __future__ import annotations

import math

import numpy as np


def lambda_pm(alpha: float, E0: float, E0d: float, C0: float):
    """Both roots lambda_-, lambda_+ of the energy constraint (Eq. 2.14).

    The discriminant vanishes at alpha = alpha_max, where rounding can make it
    slightly negative; it is clamped at zero there."""
    b = (alpha * C0 - 2.0 * E0) / (2.0 * alpha * E0)
    disc = b * b - (alpha * E0d - C0) / (alpha * E0)
    s = math.sqrt(max(0.0, disc))
    return b - s, b + s


def alpha_max(E0: float, E0d: float, C0: float) -> float:
    """Largest step with real lambda (Eq. 2.15).  By Cauchy-Schwarz the bracket
    is >= 0, with equality when u_dagger is parallel to u (the optimality
    condition lambda u0 = u_dagger); a bracket below 1e-12 of E0d/E0 is taken as
    that case (rounding) and returns inf."""
    d = E0d / E0 - C0 * C0 / (4.0 * E0 * E0)
    return math.inf if d <= 1e-12 * (E0d / E0) else 1.0 / math.sqrt(d)


def admissible_constraints(o, m: int, k: int) -> np.ndarray:
    """Rows of the linear constraints defining V for mode (m, k) != (0, 0),
    acting on x = [u_r, u_theta, u_z] (3 Nr): the three wall values and the
    discrete divergence D_r u_r + (i m / r) u_theta + i k_z u_z at every r_j,
    D_r = D1 (parity of m + 1) + 1/r."""
    nr = o.p.nr
    r = o.r
    Dr = o.d1(m + 1) + np.diag(1.0 / r)
    C = np.zeros((nr + 3, 3 * nr), np.complex128)
    for c in range(3):
        C[c, c * nr] = 1.0
    C[3:, :nr] = Dr
    C[3:, nr:2 * nr] = np.diag(1j * m / r)
    C[3:, 2 * nr:] = np.diag(1j * o.kz[k] * np.ones(nr))
    return C


def project_admissible(o, g: np.ndarray) -> np.ndarray:
    """Orthogonal projection onto V in the energy inner product (weights W_j
    per radial point; the Fourier weights are constant within a mode):
    x - W^-1 C^H (C W^-1 C^H)^-1 C x per mode, the mean mode and the
    Hermitian k = 0 plane handled by their own (diagonal) constraints."""
    p = o.p
    nr = p.nr
    out = g.astype(np.complex128).copy()
    # Hermitian k = 0 plane: average u(m) and conj u(-m)
    for i, m in enumerate(o.m):
        if m >= 0:
            j = p.M - m
            a = 0.5 * (out[:, :, i, 0] + np.conj(out[:, :, j, 0]))
            out[:, :, i, 0] = a
            out[:, :, j, 0] = np.conj(a)
    winv = np.tile(1.0 / o.W, 3)
    for i, m in enumerate(o.m):
        for k in range(p.K + 1):
            x = out[:, :, i, k].reshape(-1)
            if m == 0 and k == 0:
                x[:nr] = 0.0                      # u_r = 0
                x[nr] = 0.0                       # u_theta(wall) = 0
                uz = x[2 * nr:]
                uz[0] = 0.0
                uz -= np.dot(o.W, uz) / np.sum(o.W[1:]) * (np.arange(nr) > 0)  # zero flux
            else:
                C = admissible_constraints(o, m, k)
                S = C @ (winv[:, None] * C.conj().T)
                x = x - winv * (C.conj().T @ np.linalg.solve(S, C @ x))
            out[:, :, i, k] = x.reshape(3, nr)
    return out


def optimise(o, u0: np.ndarray, t0: float, nsteps: int, E0: float, max_iter: int, tol: float = 1e-8,
             max_halvings: int = 60, continuous: bool = False, alpha_frac: float = 1.0):
    """Adjoint looping from u0 (rescaled to E0).  Returns (u, history, info):
    history[s] is G after s accepted updates; info counts gradients (forward +
    adjoint sweeps) and forward-only gain evaluations of the line search.  With
    continuous, the gradients come from the continuous adjoint equations.
    alpha_frac scales the first trial step of each line search: 1 is the
    paper's alpha_max; a smaller fraction keeps the discriminant of Eq. 2.14
    away from zero (a conditioning choice for comparisons, not the method)."""
    grad = o.gradient_continuous if continuous else o.gradient
    u = o.scale_to(project_admissible(o, u0), E0)
    ET, g = grad(u, t0, nsteps)
    g = project_admissible(o, g)
    G = ET / o.energy(u)
    hist = [G]
    info = {"gradients": 1, "forward_evals": 0, "converged": False, "rel_change": math.nan}
    for _ in range(max_iter):
        ud = -g
        E0d = o.energy(ud)
        C0 = o.inner(u, ud)
        a = alpha_max(E0, E0d, C0)
        if not math.isfinite(a):
            info["converged"] = True
            break
        a *= alpha_frac
        accepted = None
        for _h in range(max_halvings):
            lam = lambda_pm(a, E0, E0d, C0)[1]
            un = (1.0 + lam * a) * u - a * ud
            with np.errstate(all="ignore"):
                Gn = o.energy(o.forward(un, t0, nsteps)) / o.energy(un)
            info["forward_evals"] += 1
            R = abs(Gn - G) / abs(Gn) if math.isfinite(Gn) else math.inf
            if math.isfinite(Gn) and Gn > G:
                accepted = (un, Gn, R)
                break
            if R < tol:
                break
            a *= 0.5
        if accepted is None:
            info["converged"] = True
            break
        u, Gn, R = accepted
        ET, g = grad(u, t0, nsteps)
        g = project_admissible(o, g)
        info["gradients"] += 1
        G = ET / o.energy(u)
        hist.append(G)
        info["rel_change"] = R
        if R < tol:
            info["converged"] = True
            break
    return u, hist, info
