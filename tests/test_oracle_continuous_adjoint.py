"""Pins of the continuous-adjoint oracle (Eq. 2.9-2.11 integrated backward with
the predictor-corrector of the forward step).

* no base flow, vanishing amplitude: the adjoint of the Stokes operator is the
  operator itself, and the backward sweep repeats the forward arithmetic, so
  w(0) = F^(2N) u0 exactly;
* the base-flow part of the adjoint forcing is the exact adjoint, in the energy
  inner product, of the forward base-flow terms: <L u, w> = <u, L* w>;
* consistency: the continuous gradient and the exact discrete gradient, both
  projected onto admissible fields, approach each other under radial
  refinement (they are two discretisations of the same derivative).
"""
import math

import numpy as np

from oracle import adjoint_looping as al
from oracle import pipe_oracle as po
from paper_2509_10103_gb300 import synth


def test_stokes_backward_sweep_repeats_the_forward_map():
    o = po.Oracle(po.Params(nr=12, M=2, K=3, Lz=6.0, Re=100.0, dt=0.01, Wo=8.0, A=0.0, base=False))
    p = o.p
    u0 = o.scale_to(synth.random_field(o.r, p.M, p.K, p.Lz, seed=2), 1e-60)
    N = 5
    _, g = o.gradient_continuous(u0, 0.0, N)
    ref = o.forward(o.forward(u0, 0.0, N), N * p.dt, N)
    assert np.abs(g - ref).max() <= 1e-13 * np.abs(ref).max()


def test_adjoint_base_flow_terms_are_the_transpose_of_the_forward_ones():
    o = po.Oracle(po.Params(nr=12, M=3, K=4, Lz=7.0, Re=1500.0, dt=0.01, Wo=6.0, A=0.8))
    p = o.p
    u = synth.random_field(o.r, p.M, p.K, p.Lz, seed=3)
    w = synth.random_field(o.r, p.M, p.K, p.Lz, seed=4)
    zero = np.zeros_like(u)
    t = 2.3
    eps = 1e-30  # vanishing amplitude: the forward quadratic term drops out
    Lu = o.nonlinear(eps * u, t) / eps
    Lsw = o.nonlinear_adj(w, zero, t)                   # adjoint forcing about u = 0: base-flow part only
    lhs, rhs = o.inner(Lu, w), o.inner(u, Lsw)
    assert abs(lhs - rhs) <= 1e-12 * math.sqrt(o.inner(Lu, Lu) * o.inner(w, w))


def _projected_gap(nr):
    o = po.Oracle(po.Params(nr=nr, M=2, K=3, Lz=6.0, Re=500.0, dt=0.01, Wo=8.0, A=1.0))
    p = o.p
    u0 = o.scale_to(al.project_admissible(o, synth.random_field(o.r, p.M, p.K, p.Lz, seed=2)), 1e-3)
    N = 10
    ETc, gc = o.gradient_continuous(u0, 0.0, N)
    ETd, gd = o.gradient(u0, 0.0, N)
    assert ETc == ETd  # same forward sweep
    gc, gd = al.project_admissible(o, gc), al.project_admissible(o, gd)
    return math.sqrt(o.inner(gc - gd, gc - gd) / o.inner(gd, gd))


def test_continuous_gradient_converges_to_the_discrete_one_under_refinement():
    e16, e24 = _projected_gap(16), _projected_gap(24)
    assert e16 < 0.03 and e24 < e16 / 1.5
