"""Seeded synthetic initial perturbations u0 for the pipe-flow gradient.

This module builds inputs only.  It holds none of the solver's arithmetic: no
finite differences, no quadrature, no transforms, no time stepping.  The radial
points are passed in by the caller (each side computes its own grid), and the
field is evaluated there from closed-form polynomial potentials.  Scaling to a
prescribed energy E0 is left to the caller because the discrete energy norm is
part of the method.

Construction (poloidal-toroidal potentials, exactly solenoidal in the
continuum and zero at the wall r = 1):

    psi = (1 - r^2)^2 r^|m| P1(r^2),   phi = (1 - r^2)^3 r^|m| P2(r^2)
    u   = curl(psi e_z) + curl curl(phi e_z)

For one Fourier mode exp(i m theta + i kz z) this is

    u_r     = (i m / r) psi + i kz phi'
    u_theta = -psi' - (m kz / r) phi
    u_z     = -(phi'' + phi'/r - m^2 phi / r^2)

which are evaluated term by term on the monomials of psi and phi, so no
negative powers of r appear.  P1, P2 are seeded random polynomials in r^2.
The k = 0 plane is Hermitian, u(-m, 0) = conj u(m, 0), so the physical field
is real.  Layout of the result: complex128 [3][Nr][2M+1][K+1], components
(u_r, u_theta, u_z), m = -M..M, k = 0..K, kz = 2 pi k / Lz.

Recipes (the workloads of the paper's runs, Sections 3-4 and Appendix A):
  random_field     - every mode, amplitude exp(-sqrt(m^2 + k^2) / decay)
  localised_field  - a random low-mode field times a Gaussian envelope of
                     width sigma in z centred at Lz/2 (axially localised seed)
  oblique_field    - the m = +-1 pair at one axial wavenumber (oblique waves,
                     Appendix A.2: structures of axial length 1.25 radii)
"""
from __future__ import annotations

import numpy as np

__all__ = ["random_field", "localised_field", "oblique_field", "mode_field", "single_mode"]

_POLY_DEG = 2  # degree of P1, P2 in r^2


def _potential_monomials(m: int, base_pow: int, pcoef: np.ndarray) -> np.ndarray:
    """Coefficients (ascending powers of r) of (1-r^2)^base_pow r^|m| P(r^2)."""
    am = abs(m)
    # (1 - r^2)^base_pow in powers of r^2
    w = np.array([1.0 + 0j])
    for _ in range(base_pow):
        w = np.convolve(w, np.array([1.0, -1.0]))
    q = np.convolve(w, pcoef)  # polynomial in r^2
    out = np.zeros(am + 2 * (len(q) - 1) + 1, dtype=np.complex128)
    out[am::2] = q
    return out


def _eval_terms(coef: np.ndarray, r: np.ndarray, factor) -> np.ndarray:
    """sum_n coef[n] * factor(n) * r^(n - shift) where factor returns (value, shift)."""
    res = np.zeros(r.shape, dtype=np.complex128)
    for n, c in enumerate(coef):
        if c == 0:
            continue
        f, shift = factor(n)
        if f == 0:
            continue
        p = n - shift
        if p < 0:
            raise ValueError("negative power in potential evaluation")
        res += c * f * r ** p
    return res


def mode_field(r: np.ndarray, m: int, kz: float, psi: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Velocity (3, Nr) of one mode from potential monomial coefficients psi, phi."""
    r = np.asarray(r, dtype=np.float64)
    ur = (1j * m) * _eval_terms(psi, r, lambda n: (1.0, 1)) if m != 0 else np.zeros(r.shape, np.complex128)
    ur = ur + (1j * kz) * _eval_terms(phi, r, lambda n: (float(n), 1))
    ut = -_eval_terms(psi, r, lambda n: (float(n), 1))
    if m != 0:
        ut = ut - (m * kz) * _eval_terms(phi, r, lambda n: (1.0, 1))
    uz = -_eval_terms(phi, r, lambda n: (float(n * n - m * m), 2))
    return np.stack([ur, ut, uz])


def _rand_poly(rng: np.random.Generator, real: bool) -> np.ndarray:
    if real:
        return rng.standard_normal(_POLY_DEG + 1) + 0j
    return rng.standard_normal(_POLY_DEG + 1) + 1j * rng.standard_normal(_POLY_DEG + 1)


def _assemble(r, M, K, Lz, coeffs) -> np.ndarray:
    """coeffs: dict (m, k) -> (psi_monomials, phi_monomials) for k >= 0."""
    nr = len(r)
    u = np.zeros((3, nr, 2 * M + 1, K + 1), dtype=np.complex128)
    for (m, k), (psi, phi) in coeffs.items():
        kz = 2.0 * np.pi * k / Lz
        u[:, :, m + M, k] = mode_field(r, m, kz, psi, phi)
    # exact Hermitian symmetry of the k = 0 plane
    for m in range(1, M + 1):
        u[:, :, M - m, 0] = np.conj(u[:, :, M + m, 0])
    u[:, :, M, 0] = u[:, :, M, 0].real
    return u


def random_field(r, M: int, K: int, Lz: float, seed: int = 0, decay: float = 4.0) -> np.ndarray:
    """Every mode excited, amplitude exp(-sqrt(m^2 + k^2) / decay) (integer indices)."""
    rng = np.random.default_rng(seed)
    coeffs = {}
    for k in range(K + 1):
        for m in range(-M, M + 1):
            if k == 0 and m < 0:
                continue
            amp = np.exp(-np.sqrt(m * m + k * k) / decay)
            real = (k == 0 and m == 0)
            p1, p2 = _rand_poly(rng, real), _rand_poly(rng, real)
            coeffs[(m, k)] = (amp * _potential_monomials(m, 2, p1), amp * _potential_monomials(m, 3, p2))
    return _assemble(r, M, K, Lz, coeffs)


def localised_field(r, M: int, K: int, Lz: float, seed: int = 0, sigma: float = 3.0,
                    m_low: int = 3, kz_low: float = 2.0, decay: float = 4.0) -> np.ndarray:
    """Random low-mode field times exp(-(z - Lz/2)^2 / (2 sigma^2)).

    The product in z is a convolution of axial spectra; the envelope's Fourier
    coefficients are those of the periodised Gaussian, truncated to |k| <= K.
    """
    rng = np.random.default_rng(seed)
    kc = max(1, int(np.ceil(kz_low * Lz / (2.0 * np.pi))))
    mc = min(m_low, M)
    # underlying real low-mode field c[(m, k0)], k0 in [-kc, kc], Hermitian in (m, k0)
    low = {}
    for k0 in range(0, kc + 1):
        for m in range(-mc, mc + 1):
            if k0 == 0 and m < 0:
                continue
            amp = np.exp(-np.sqrt(m * m + k0 * k0) / decay)
            real = (k0 == 0 and m == 0)
            low[(m, k0)] = (amp * _rand_poly(rng, real), amp * _rand_poly(rng, real))
    for (m, k0), (p1, p2) in list(low.items()):
        if (-m, -k0) not in low:
            low[(-m, -k0)] = (np.conj(p1), np.conj(p2))
    def ghat(k):
        kz = 2.0 * np.pi * k / Lz
        return (sigma * np.sqrt(2.0 * np.pi) / Lz) * np.exp(-0.5 * (kz * sigma) ** 2) * np.exp(-1j * kz * Lz / 2.0)
    coeffs = {}
    for k in range(K + 1):
        for m in range(-mc, mc + 1):
            if k == 0 and m < 0:
                continue
            p1 = np.zeros(_POLY_DEG + 1, np.complex128)
            p2 = np.zeros(_POLY_DEG + 1, np.complex128)
            for k0 in range(-kc, kc + 1):
                if (m, k0) in low:
                    g = ghat(k - k0)
                    p1 = p1 + g * low[(m, k0)][0]
                    p2 = p2 + g * low[(m, k0)][1]
            coeffs[(m, k)] = (_potential_monomials(m, 2, p1), _potential_monomials(m, 3, p2))
    return _assemble(r, M, K, Lz, coeffs)


def oblique_field(r, M: int, K: int, Lz: float, seed: int = 0, wavelength: float = 1.25,
                  noise: float = 1e-3) -> np.ndarray:
    """Equal-amplitude m = +1 and m = -1 waves at the axial index nearest Lz/wavelength,
    plus a weak random background (relative amplitude `noise`)."""
    rng = np.random.default_rng(seed)
    k_ob = int(round(Lz / wavelength))
    if k_ob > K or M < 1:
        raise ValueError("oblique wave outside the resolved modes")
    base = random_field(r, M, K, Lz, seed=seed + 7919, decay=4.0) * noise
    p1 = _rand_poly(rng, False)
    p2 = _rand_poly(rng, False)
    coeffs = {}
    for m in (1, -1):
        coeffs[(m, k_ob)] = (_potential_monomials(m, 2, p1), _potential_monomials(m, 3, p2))
    wave = _assemble(r, M, K, Lz, coeffs)
    return base + wave


def single_mode(r, m: int, k: int, Lz: float, seed: int = 0) -> np.ndarray:
    """Velocity profile (3, Nr) of one random solenoidal mode (m, k); real
    potentials for the mode (0, 0)."""
    rng = np.random.default_rng(seed)
    real = (m == 0 and k == 0)
    psi = _potential_monomials(m, 2, _rand_poly(rng, real))
    phi = _potential_monomials(m, 3, _rand_poly(rng, real))
    return mode_field(r, m, 2.0 * np.pi * k / Lz, psi, phi)
