"""Assembled global stiffness (oracle; test infrastructure only).

K(rho) = sum_e E_e A_e^T K0 A_e with the SIMP modulus of Eq. K_mod read as
E_e = Emin + rho_e^p (E0 - Emin), i.e. K_min = (Emin/E0) K0 (the paper's
K_min is "minimum stiffness" and is not defined further).

Dirichlet conditions u_d = 0 are imposed by zeroing the fixed rows and
columns and putting 1 on their diagonal; the load at fixed DOFs is zeroed.
The resulting system has the same free-DOF solution as the constrained
problem and u = 0 at fixed DOFs.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import element_dofs, n_nodes


def simp_modulus(rho, E0=1.0, Emin=1e-9, penal=3.0):
    """E(rho) = Emin + rho^p (E0 - Emin)  (Eq. K_mod with K_min = (Emin/E0) K0)."""
    rho = np.asarray(rho, dtype=np.float64)
    return Emin + rho ** penal * (E0 - Emin)


def assemble(dims, E_elem, K0) -> sp.csr_matrix:
    """Global K = sum_e E_e A_e^T K0 A_e, no boundary conditions (CSR, FP64)."""
    edof = element_dofs(dims)
    nel = edof.shape[0]
    ndof = 3 * n_nodes(dims)
    E_elem = np.asarray(E_elem, dtype=np.float64).reshape(nel)
    rows = np.repeat(edof, 24, axis=1).ravel()
    cols = np.tile(edof, (1, 24)).ravel()
    vals = (E_elem[:, None] * K0.ravel()[None, :]).ravel()
    idx_t = np.int32 if ndof < 2**31 - 1 else np.int64
    K = sp.coo_matrix((vals, (rows.astype(idx_t), cols.astype(idx_t))), shape=(ndof, ndof))
    return K.tocsr()


def apply_dirichlet(K: sp.csr_matrix, fixed) -> sp.csr_matrix:
    """Zero fixed rows and columns, unit diagonal on fixed DOFs."""
    fixed = np.asarray(fixed).astype(bool)
    free = (~fixed).astype(np.float64)
    Pf = sp.diags(free)
    Kd = (Pf @ K @ Pf).tocsr()
    Kd = Kd + sp.diags(fixed.astype(np.float64))
    Kd.eliminate_zeros()
    return Kd.tocsr()


def constrained_system(dims, E_elem, K0, fixed, f):
    """(K with Dirichlet rows, f with fixed entries zeroed)."""
    K = apply_dirichlet(assemble(dims, E_elem, K0), fixed)
    f = np.where(np.asarray(fixed).astype(bool), 0.0, np.asarray(f, dtype=np.float64))
    return K, f
