"""Writes cfg2_oracle_100steps.json: the FP64 oracle's gradient of the final
perturbation energy over the first 100 steps of the localised-perturbation
workload (nr=48, |m|<=15, |k|<=47, Lz=50, Re=2500, A=1, Wo=8, dt=0.005,
tau0=0, E0=1e-5, localised seed 0 with sigma=3).

Only the oracle (and the seeded input generator) is called.  A full gradient
field is 3.4 MB, so the file keeps what a parity test can compare without
it: the gain, the energy norm of the gradient, its energy inner products with
eight seeded directions, and 320 sampled coefficients (256 at seeded
positions, the 64 largest in magnitude).  The oracle needs several
minutes of CPU time for this, which is why the values are stored.

It also records how far the oracle's result moves under its own rounding:
the same gradient with every dense per-mode stage map formed as inv(A) @ B
instead of solve(A, B) (equal in exact arithmetic).  Over 100 steps at this
resolution the two differ by about 1e-10 of the gradient's largest value,
so that spread, not the parity of the CUDA path, sets the floor of a
max-norm comparison here.

Usage: python tests/golden/make_cfg2_oracle.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pipe_oracle as po  # noqa: E402
from paper_2509_10103_gb300 import synth  # noqa: E402

CFG = dict(nr=48, M=15, K=47, Lz=50.0, Re=2500.0, dt=0.005, Wo=8.0, A=1.0)
E0 = 1e-5
NSTEPS = 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg2_oracle_100steps.json")


def directions(o, n=8):
    return [synth.random_field(o.r, o.p.M, o.p.K, o.p.Lz, seed=200 + s) for s in range(n)]


def sample_indices(shape, n=256, seed=7):
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(0, d)) for d in shape) for _ in range(n)]


def main():
    o = po.Oracle(po.Params(**CFG))
    u0 = o.scale_to(synth.localised_field(o.r, CFG["M"], CFG["K"], CFG["Lz"], seed=0), E0)
    ET, g = o.gradient(u0, 0.0, NSTEPS)
    solve = np.linalg.solve
    np.linalg.solve = lambda a, b: np.linalg.inv(a) @ b  # the second, equally valid rounding of the maps
    try:
        o2 = po.Oracle(po.Params(**CFG))
        ET2, g2 = o2.gradient(u0, 0.0, NSTEPS)
    finally:
        np.linalg.solve = solve
    idx = sample_indices(g.shape)
    top = np.argsort(np.abs(g).ravel())[::-1][:64]
    idx += [tuple(int(i) for i in np.unravel_index(t, g.shape)) for t in top]
    out = {
        "config": CFG, "E0": E0, "nsteps": NSTEPS, "tau0": 0.0, "seed": 0, "sigma": 3.0,
        "gain": ET / o.energy(u0),
        "grad_norm2": o.inner(g, g),
        "grad_max": float(np.abs(g).max()),
        "oracle_spread": {"gain_rel": abs(ET2 / ET - 1),
                          "grad_maxnorm_rel": float(np.abs(g2 - g).max() / np.abs(g).max()),
                          "grad_energy_norm_rel": float(np.sqrt(o.inner(g2 - g, g2 - g) / o.inner(g, g)))},
        "dir_seeds": [200 + s for s in range(8)],
        "grad_dot_dirs": [o.inner(g, v) for v in directions(o)],
        "samples": [[list(i), [float(g[i].real), float(g[i].imag)]] for i in idx],
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(OUT, out["gain"])


if __name__ == "__main__":
    main()
