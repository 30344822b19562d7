"""Optimality-criteria update (oracle; test infrastructure only).

Eq. OCUp1 / Eq. bisect as printed are garbled (the move-limit bounds lack
the current density; an extra exponent q "typically 2" is mentioned).  The
reading used here is the standard OC step of compliance topology
optimisation with the filter chain rule:

    dc~ = H^T dc,  dv~ = H^T 1                      (H the density filter)
    B_e = max(-dc~_e, 1e-30) / (lambda dv~_e)
    x_new = max(0, max(x - m, min(1, min(x + m, x B^eta)))),   eta = 1/2, q = 1

with lambda found by bisection (the paper names bisection without bounds or
tolerance): l1 = 0, l2 = 1e9; while (l2 - l1)/(l1 + l2) > 1e-9:
lambda = (l1 + l2)/2, evaluate x_new(lambda), and if the mean filtered
density mean(H x_new) exceeds volfrac set l1 = lambda, else l2 = lambda.
The returned design is x_new of the last lambda evaluated, and the change is
||x_new - x||_inf (the stopping quantity named after Eq. bisect).

With the paper's sensitivity filter the design is its own physical density:
oc_update_unfiltered takes already filtered sensitivities, B_e =
max(-dc_e, 1e-30) / lambda, and bisects on mean(x_new) against volfrac, with
the same bounds, tolerance and clamps.
"""
from __future__ import annotations

import numpy as np

from .filter import density_filter, density_filter_T


def oc_update(x, dc, dims, r, volfrac, move=0.2, eta=0.5, l1=0.0, l2=1e9, tol=1e-9):
    """Returns (x_new, change, lambda_last, bisection_steps)."""
    x = np.asarray(x, dtype=np.float64)
    dct = density_filter_T(dc, dims, r)
    dvt = density_filter_T(np.ones_like(x), dims, r)
    num = np.maximum(-dct, 1e-30)
    xnew = x.copy()
    lmid = 0.5 * (l1 + l2)
    steps = 0
    while (l2 - l1) / (l1 + l2) > tol:
        lmid = 0.5 * (l1 + l2)
        cand = x * (num / (lmid * dvt)) ** eta
        xnew = np.maximum(0.0, np.maximum(x - move, np.minimum(1.0, np.minimum(x + move, cand))))
        if density_filter(xnew, dims, r).mean() > volfrac:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    return xnew, float(np.max(np.abs(xnew - x))), lmid, steps


def oc_update_unfiltered(x, dc, volfrac, move=0.2, eta=0.5, l1=0.0, l2=1e9, tol=1e-9, passive=None):
    """OC step on a design without density filter (sensitivities filtered by
    Eq. sensitivity filter beforehand).  passive (optional, per element):
    0 active, 1 passive solid (x = 1), 2 passive void (x = 0); passive
    elements take their value and the volume fraction is that of the active
    elements (Sec. 5, Examples 2 and 4).  Returns (x_new, change,
    lambda_last, bisection_steps)."""
    x = np.asarray(x, dtype=np.float64)
    num = np.maximum(-np.asarray(dc, dtype=np.float64), 1e-30)
    pas = np.zeros(x.size, dtype=np.uint8) if passive is None else np.asarray(passive, dtype=np.uint8)
    active = pas == 0
    xnew = x.copy()
    lmid = 0.5 * (l1 + l2)
    steps = 0
    while (l2 - l1) / (l1 + l2) > tol:
        lmid = 0.5 * (l1 + l2)
        cand = x * (num / lmid) ** eta
        xnew = np.maximum(0.0, np.maximum(x - move, np.minimum(1.0, np.minimum(x + move, cand))))
        xnew[pas == 1] = 1.0
        xnew[pas == 2] = 0.0
        if xnew[active].mean() > volfrac:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    return xnew, float(np.max(np.abs(xnew - x))), lmid, steps
