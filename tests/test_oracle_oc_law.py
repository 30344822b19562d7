"""Pin of the OC update law (Eqs. OCUp1, bisect) from a different principle.

The printed update is garbled (bounds without the current density, an extra
exponent q), so the oracle takes the reading x_new = clamp(x B^(1/2)) with
q = 1.  That reading is pinned here without re-typing it: the OC step of
compliance minimisation is the exact minimiser of the convex separable
subproblem obtained by linearising the compliance in the reciprocal
variables y_e = 1/x_e (the CONLIN approximation, Fleury 1989),

    minimise   sum_e a_e / x'_e,        a_e = -dc~_e x_e^2 > 0,
    subject to sum_e dv~_e x'_e = N volfrac,     (the linear volume, H^T 1 = dv~)
               max(0, x_e - m) <= x'_e <= min(1, x_e + m).

The subproblem is solved by a general constrained optimiser (SLSQP); the
oracle's bisection result must agree with it on every element, clamped or
not.  A law with eta = 1, the paper's q = 2 applied to the unclamped value,
or a volume derivative without the filter transpose gives another minimiser
(tests/test_oracle_planted.py plants all three).
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import synth
from oracle import filter as flt, oc


def conlin_step(x, dct, dvt, target_sum, move):
    """Minimiser of the reciprocal-variable subproblem above (scipy SLSQP)."""
    a = -dct * x * x
    lo = np.maximum(0.0, x - move)
    hi = np.minimum(1.0, x + move)
    scale = 1.0 / a.sum()                        # objective of order one
    res = minimize(lambda y: scale * np.sum(a / y), np.clip(x, lo, hi),
                   jac=lambda y: -scale * a / (y * y), method="SLSQP",
                   bounds=list(zip(lo, hi)),
                   constraints=[{"type": "eq", "fun": lambda y: (dvt @ y - target_sum) / len(y),
                                 "jac": lambda y: dvt / len(y)}],
                   options={"ftol": 1e-16, "maxiter": 2000})
    assert res.success, res.message
    return res.x


def _filtered_case():
    dims = (6, 4, 3)
    r, vf, move = 2.0, 0.45, 0.1
    x = synth.uniform_field(dims, 41, 0.3, 0.8)
    dc = -synth.uniform_field(dims, 42, 0.05, 20.0)
    return dims, r, vf, move, x, dc


def oc_law_error(update, dims, r, vf, move, x, dc):
    """max |x_new - x_conlin| for an OC update with the oracle's signature."""
    xn = update(x, dc, dims, r, vf, move)[0]
    dct = flt.density_filter_T(dc, dims, r)
    dvt = flt.density_filter_T(np.ones_like(x), dims, r)
    ref = conlin_step(x, dct, dvt, vf * x.size, move)
    return np.abs(xn - ref).max(), xn, x, move


def test_oc_update_is_the_conlin_minimiser():
    err, xn, x, move = oc_law_error(oc.oc_update, *_filtered_case())
    inside = (xn > np.maximum(0.0, x - move) + 1e-6) & (xn < np.minimum(1.0, x + move) - 1e-6)
    assert inside.sum() >= 10 and (~inside).sum() >= 5      # both branches occur
    assert err < 1e-6


def test_oc_update_unfiltered_is_the_conlin_minimiser():
    dims = (5, 4, 3)
    vf, move = 0.5, 0.15
    x = synth.uniform_field(dims, 43, 0.3, 0.8)
    dc = -synth.uniform_field(dims, 44, 0.2, 3.0)
    xn = oc.oc_update_unfiltered(x, dc, vf, move)[0]
    ref = conlin_step(x, dc, np.ones_like(x), vf * x.size, move)
    inside = (xn > np.maximum(0.0, x - move) + 1e-6) & (xn < np.minimum(1.0, x + move) - 1e-6)
    assert inside.sum() >= 10
    assert np.abs(xn - ref).max() < 1e-6


def test_conlin_solver_recovers_a_known_minimiser():
    """The pin's own solver: with a_e = c dv~_e t_e^2 the unconstrained
    stationary point of sum a/x' + lambda dv~.x' is x' = t sqrt(c/lambda);
    choosing the volume so that lambda = c puts the minimiser at t exactly."""
    rng = np.random.default_rng(7)
    n = 40
    t = rng.uniform(0.3, 0.7, n)
    dvt = rng.uniform(0.5, 1.5, n)
    x = np.full(n, 0.5)
    dct = -(2.0 * dvt * t * t) / (x * x)          # a_e = 2 dv~_e t_e^2
    got = conlin_step(x, dct, dvt, dvt @ t, move=0.3)
    assert np.abs(got - t).max() < 1e-7
