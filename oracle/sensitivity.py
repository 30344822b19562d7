"""Compliance and its adjoint sensitivity (oracle; test infrastructure only).

Compliance c = f^T u (Eq. compliance objective).  The adjoint equation
K u* = dc/du = f has the solution u* = u (self-adjoint), so Eq. sensitivity
becomes, per element, with the SIMP law of Eq. K_mod
(K_e = (Emin + rho_e^p (E0 - Emin)) K0):

    dc/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T K0 u_e.

The energy identity c = f^T u = u^T K u = sum_e E_e u_e^T K0 u_e holds at
the exact solution and is used as a check.

Design-dependent gravity load (Sec. 5, Example 4: a load proportional to
the material present): element e of density rho_e carries the weight
w rho_e in -z, a constant body force whose consistent nodal load on the
trilinear brick is one eighth at each corner, so f(rho) = f_ext +
sum_e rho_e g_e with g_e = -(w/8) e_z at the 8 corners.  Then
dc/drho_e = 2 u_e^T g_e - p rho_e^(p-1) (E0 - Emin) u_e^T K0 u_e
(c = f^T u with K u = f: dc = 2 u^T df - u^T dK u).
"""
from __future__ import annotations

import numpy as np

from .grid import element_dofs


def compliance(f, u) -> float:
    return float(np.dot(f, u))


def element_energy(u, dims, K0) -> np.ndarray:
    """u_e^T K0 u_e for every element."""
    ue = np.asarray(u, dtype=np.float64)[element_dofs(dims)]
    return np.einsum("ea,ab,eb->e", ue, K0, ue)


def sensitivity(rho, se, E0=1.0, Emin=1e-9, penal=3.0) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    return -penal * rho ** (penal - 1.0) * (E0 - Emin) * se


def gravity_load(dims, rho, w, f_ext=None) -> np.ndarray:
    """f_ext + sum_e rho_e g_e (no Dirichlet masking)."""
    from .grid import element_nodes, n_nodes
    rho = np.asarray(rho, dtype=np.float64)
    f = np.zeros(3 * n_nodes(dims)) if f_ext is None else np.array(f_ext, dtype=np.float64)
    nodes = element_nodes(dims)
    for a in range(8):
        np.add.at(f, 3 * nodes[:, a] + 2, -w / 8.0 * rho)
    return f


def gravity_sensitivity_term(dims, u, w) -> np.ndarray:
    """2 u_e^T g_e = -(w/4) * (sum of u_z over the 8 corners of e)."""
    from .grid import element_nodes
    u = np.asarray(u, dtype=np.float64)
    return -(w / 4.0) * u[3 * element_nodes(dims) + 2].sum(axis=1)
