"""Resolution and growth diagnostics from the per-mode energy spectrum that
pnop_mode_energy returns (shape (2, 2M+1, K+1): cross-section and axial parts
of each stored mode m = -M..M, k = 0..K; stored modes with k > 0 carry their
conjugate partner (-m, -k) as well).

* e_M, e_K (Section 2.4): the energy of the highest azimuthal mode m = M,
  respectively axial mode k = K, summed over the other index of the full
  spectrum (k = -K..K, respectively m = -M..M), over E0.  The paper keeps both
  below 1e-8.
* G_(r,theta) and G_z (Section 3): the cross-section and axial parts of the
  energy growth E(t)/E0.
"""
from __future__ import annotations

import numpy as np


def resolution_measures(spectrum: np.ndarray, E0: float):
    """(e_M, e_K) from a (2, 2M+1, K+1) spectrum."""
    E = np.asarray(spectrum).sum(axis=0)
    nm, nk = E.shape
    M, K = (nm - 1) // 2, nk - 1
    # full-spectrum energy of (M, k) for k = -K..K: the stored (M, 0), and half of
    # each stored (M, k) and (-M, k), k > 0 (each holds e(m, k) + e(-m, -k))
    e_M = E[2 * M, 0] + 0.5 * (E[2 * M, 1:].sum() + E[0, 1:].sum()) if M > 0 else E[0].sum()
    # full-spectrum energy of (m, K) for m = -M..M: half of each stored (m, K), K > 0
    e_K = 0.5 * E[:, K].sum() if K > 0 else E[:, 0].sum()
    return float(e_M / E0), float(e_K / E0)


def component_gains(spectrum: np.ndarray, E0: float):
    """(G_(r,theta), G_z): cross-section and axial energy over E0."""
    s = np.asarray(spectrum)
    return float(s[0].sum() / E0), float(s[1].sum() / E0)
