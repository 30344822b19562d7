"""Compliance and its adjoint sensitivity (oracle; test infrastructure only).

Compliance c = f^T u (Eq. compliance objective).  The adjoint equation
K u* = dc/du = f has the solution u* = u (self-adjoint), so Eq. sensitivity
becomes, per element, with the SIMP law of Eq. K_mod
(K_e = (Emin + rho_e^p (E0 - Emin)) K0):

    dc/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T K0 u_e.

The energy identity c = f^T u = u^T K u = sum_e E_e u_e^T K0 u_e holds at
the exact solution and is used as a check.
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
