"""Density filter and its transpose (oracle; test infrastructure only).

Weights follow Eq. Neighbourhood, w(x_i, x_e) = r - ||x_i - x_e|| for
||x_i - x_e|| <= r and 0 beyond, over the neighbourhood of Eq. NB_dist,
with x the element centres in element units.  The paper applies these
weights in a sensitivity filter (Eq. sensitivity filter); the hot path uses
them as a density filter

    rho~_e = sum_i w_ei rho_i / S_e,   S_e = sum_i w_ei,

with the sums over elements inside the domain (the neighbourhood is cut at
the boundary and S_e normalises over the elements that remain).  Its
transpose, needed by the chain rule dc/drho = H^T dc/drho~, is
(H^T g)_i = sum_e w_ei g_e / S_e.

The paper's own filter (Eq. sensitivity filter) smooths the sensitivities
of the design itself:

    dc^_e = sum_i w_ei rho_i dc_i / (max(gamma, rho_e) S_e),

gamma > 0 small (1e-3 here; the paper leaves its value open).
"""
from __future__ import annotations

import math

import numpy as np


def offsets(r: float):
    """Integer offsets with positive weight r - |d| (|d| < r)."""
    R = int(math.ceil(r))
    out = []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = r - math.sqrt(dx * dx + dy * dy + dz * dz)
                if w > 0.0:
                    out.append((dx, dy, dz, w))
    return out


def _shift_accumulate(out3, src3, dx, dy, dz, w):
    """out[k,j,i] += w * src[k+dz, j+dy, i+dx] where both are inside the grid."""
    nz, ny, nx = src3.shape
    i0, i1 = max(0, -dx), nx - max(0, dx)
    j0, j1 = max(0, -dy), ny - max(0, dy)
    k0, k1 = max(0, -dz), nz - max(0, dz)
    if i0 >= i1 or j0 >= j1 or k0 >= k1:
        return
    out3[k0:k1, j0:j1, i0:i1] += w * src3[k0 + dz:k1 + dz, j0 + dy:j1 + dy, i0 + dx:i1 + dx]


def weight_sums(dims, r) -> np.ndarray:
    nx, ny, nz = dims
    S = np.zeros((nz, ny, nx))
    one = np.ones((nz, ny, nx))
    for dx, dy, dz, w in offsets(r):
        _shift_accumulate(S, one, dx, dy, dz, w)
    return S.ravel()


def density_filter(x, dims, r) -> np.ndarray:
    nx, ny, nz = dims
    x3 = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx)
    acc = np.zeros_like(x3)
    for dx, dy, dz, w in offsets(r):
        _shift_accumulate(acc, x3, dx, dy, dz, w)
    return acc.ravel() / weight_sums(dims, r)


def density_filter_T(g, dims, r) -> np.ndarray:
    nx, ny, nz = dims
    gs = (np.asarray(g, dtype=np.float64) / weight_sums(dims, r)).reshape(nz, ny, nx)
    acc = np.zeros_like(gs)
    for dx, dy, dz, w in offsets(r):
        _shift_accumulate(acc, gs, dx, dy, dz, w)
    return acc.ravel()


def sensitivity_filter(rho, dc, dims, r, gamma=1e-3) -> np.ndarray:
    """Eq. sensitivity filter over the same cut neighbourhoods and sums S_e."""
    nx, ny, nz = dims
    rho = np.asarray(rho, dtype=np.float64)
    t3 = (rho * np.asarray(dc, dtype=np.float64)).reshape(nz, ny, nx)
    acc = np.zeros_like(t3)
    for dx, dy, dz, w in offsets(r):
        _shift_accumulate(acc, t3, dx, dy, dz, w)
    return acc.ravel() / (np.maximum(gamma, rho) * weight_sums(dims, r))


def density_filter_bruteforce(x, dims, r) -> np.ndarray:
    """O(N^2) pure-Python loops over all element pairs (tiny grids only)."""
    nx, ny, nz = dims
    cent = [(i + 0.5, j + 0.5, k + 0.5) for k in range(nz) for j in range(ny) for i in range(nx)]
    out = []
    for ce in cent:
        num = den = 0.0
        for ci, xi in zip(cent, x):
            d = math.dist(ce, ci)
            if d <= r:
                w = r - d
                num += w * xi
                den += w
        out.append(num / den)
    return np.asarray(out)
