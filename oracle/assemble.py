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


def operator_rows(dims, nodes, E_of, u_of, K0, fixed_of=None):
    """Rows of the Dirichlet operator K~ u for a few nodes, from local data only.

    (K~ u)_n = sum over the (up to 8) elements e containing node n of
    E_e (K0 u_e) restricted to the corner of n, with fixed DOFs of u taken as
    zero and the rows of fixed DOFs replaced by u (the convention of
    apply_dirichlet).  E_of(element ids) and u_of(dof ids) / fixed_of(dof ids)
    return values for the requested ids, so the full vectors never need to
    exist (used to check very large grids at sampled nodes).
    Returns an array (len(nodes), 3).
    """
    nx, ny, nz = dims
    NX, NY = nx + 1, ny + 1
    out = np.zeros((len(nodes), 3))
    for r, n in enumerate(nodes):
        n = int(n)
        i, j, k = n % NX, (n // NX) % NY, n // (NX * NY)
        dofs_n = 3 * n + np.arange(3)
        fixed_n = fixed_of(dofs_n).astype(bool) if fixed_of is not None else np.zeros(3, bool)
        acc = np.zeros(3)
        for ez in (k - 1, k):
            for ey in (j - 1, j):
                for ex in (i - 1, i):
                    if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                        continue
                    e = ex + nx * (ey + ny * ez)
                    corners = [(ex + ax) + NX * ((ey + ay) + NY * (ez + az))
                               for az in (0, 1) for ay in (0, 1) for ax in (0, 1)]
                    edofs = (3 * np.asarray(corners)[:, None] + np.arange(3)).ravel()
                    ue = np.asarray(u_of(edofs), dtype=np.float64)
                    if fixed_of is not None:
                        ue = np.where(np.asarray(fixed_of(edofs)).astype(bool), 0.0, ue)
                    a = corners.index(n)
                    acc += float(E_of(np.array([e]))[0]) * (K0[3 * a:3 * a + 3, :] @ ue)
        u_n = np.asarray(u_of(dofs_n), dtype=np.float64)
        out[r] = np.where(fixed_n, u_n, acc)
    return out
