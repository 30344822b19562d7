"""Linear solves of K u = f (oracle; test infrastructure only).

* solve_dense: Cholesky factorisation and two triangular solves (the direct
  method of Sec. 3.1, used by Algorithm 4's "Direct solve" step) -- tiny grids.
* solve_sparse_direct: sparse LU (SuperLU) -- small grids.
* pcg: the preconditioned conjugate gradient method of Algorithm 1.  Its
  printed initialisation is garbled ("z0 = M^-1 r0 = 0"); it is read as the
  standard method: x0 = warm start (0 by default), r0 = f - K x0,
  z0 = M^-1 r0, p0 = z0.  The loop stops when ||r||_2 / ||f||_2 <= tol.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve_dense(K, f) -> np.ndarray:
    A = K.toarray() if sp.issparse(K) else np.asarray(K)
    L = np.linalg.cholesky(A)
    y = sla.solve_triangular(L, f, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def solve_sparse_direct(K, f) -> np.ndarray:
    return spla.spsolve(sp.csc_matrix(K), f)


def pcg(K, f, M_apply=None, tol=1e-10, max_it=10000, x0=None):
    """Algorithm 1 (PCG).  Returns (x, iterations, final ||r||/||f||)."""
    f = np.asarray(f, dtype=np.float64)
    nf = np.linalg.norm(f)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    if nf == 0.0:
        return np.zeros_like(f), 0, 0.0
    r = f - K @ x
    if np.linalg.norm(r) / nf <= tol:
        return x, 0, np.linalg.norm(r) / nf
    z = M_apply(r) if M_apply is not None else r.copy()
    p = z.copy()
    rz = r @ z
    it = 0
    relres = np.linalg.norm(r) / nf
    while it < max_it:
        q = K @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        relres = np.linalg.norm(r) / nf
        if relres <= tol:
            break
        z = M_apply(r) if M_apply is not None else r.copy()
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, relres
