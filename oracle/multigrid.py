"""Geometric multigrid on the brick grid (oracle; test infrastructure only).

Grid transfer (Sec. 3.2, Figs. restriction / linear interpolation and the
restriction matrix of Sec. 4.2.2).  Level l has nx/2^l x ny/2^l x nz/2^l
elements of edge 2^l.  Prolongation I_{2h}^h is trilinear nodal
interpolation (1D weights 1 at coincident nodes, 1/2 at midpoints); the
restriction is its transpose, I_h^{2h} = (I_{2h}^h)^T.  The paper prints the
1D restriction rows as (1/4)[1 2 1]; the transpose of interpolation has rows
(1/2)[1 2 1].  A positive scale only rescales the coarse correction; the
transpose is the choice for which I_h^{2h} K^h I_{2h}^h equals the coarse
rediscretisation for uniform stiffness (checked in the tests).

Homogenized coarse operators (Sec. 4.2.2 and Sec. 6): the density of a
coarse element is the mean of the densities of its eight children; the
coarse element matrix is E(rho_coarse) * 2^l K0 (3D elastic stiffness
scales linearly with the element edge).  The SIMP law is applied after
averaging the density (the paper averages "density values").

Dirichlet conditions on coarse levels: a coarse DOF is fixed iff the fine
DOF at the coincident node is fixed (injection).  The transfers are
P~ = diag(free_fine) P diag(free_coarse), R~ = P~^T.

V-cycle (Algorithm 3): pre-smooth, restrict the residual, recurse with a
zero initial iterate, prolongate and correct, post-smooth; on the coarsest
grid the problem is solved directly.  The smoother is damped Jacobi
(Sec. 3.2, damped Jacobi equation) u <- u + omega D^-1 (f - K u); the first
sweep from u = 0 is u = omega D^-1 f.  omega, and the numbers of sweeps are
not given in the paper.  The defaults are two sweeps before and after (the
same counts so that the preconditioner is symmetric) and omega = 0.35: with
theta = lambda_max(diag(K0)^-1 K0) = 5.318 (nu = 0.3), the Rayleigh quotient
u^T K u / u^T D u of any SIMP-scaled assembly is at most theta, so
omega < 2/theta = 0.376 makes the smoother convergent in the K-norm for every
density field, and the V-cycle is then symmetric positive definite for any
SPD coarse operators (homogenized or not).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .assemble import apply_dirichlet, assemble, simp_modulus
from .solve import pcg, solve_dense


def coarse_dims(dims, levels_down=1):
    f = 2 ** levels_down
    nx, ny, nz = dims
    if nx % f or ny % f or nz % f:
        raise ValueError(f"grid {dims} not divisible by {f}")
    return (nx // f, ny // f, nz // f)


def prolongation_1d(nc: int) -> sp.csr_matrix:
    """(2 nc + 1) x (nc + 1) linear interpolation along one axis."""
    rows, cols, vals = [], [], []
    for I in range(nc + 1):
        rows.append(2 * I), cols.append(I), vals.append(1.0)
    for I in range(nc):
        rows += [2 * I + 1, 2 * I + 1]
        cols += [I, I + 1]
        vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc + 1, nc + 1))


def prolongation_nodes(dims_coarse) -> sp.csr_matrix:
    """Trilinear nodal interpolation coarse -> fine (x fastest numbering)."""
    nx, ny, nz = dims_coarse
    return sp.kron(prolongation_1d(nz), sp.kron(prolongation_1d(ny), prolongation_1d(nx))).tocsr()


def prolongation_dofs(dims_coarse) -> sp.csr_matrix:
    return sp.kron(prolongation_nodes(dims_coarse), sp.identity(3)).tocsr()


def inject_fixed(dims_fine, fixed_fine) -> np.ndarray:
    """Coarse Dirichlet mask: DOF of coarse node (I,J,K) <- fine node (2I,2J,2K)."""
    nxc, nyc, nzc = coarse_dims(dims_fine)
    nx, ny, _ = dims_fine
    K, J, I = np.meshgrid(np.arange(nzc + 1), np.arange(nyc + 1), np.arange(nxc + 1), indexing="ij")
    fine_node = (2 * I.ravel()) + (nx + 1) * ((2 * J.ravel()) + (ny + 1) * (2 * K.ravel()))
    ff = np.asarray(fixed_fine).reshape(-1, 3)
    return ff[fine_node].reshape(-1).astype(np.uint8)


def homogenize_density(rho, dims) -> np.ndarray:
    """Coarse density = mean of the eight children (Sec. 4.2.2)."""
    nx, ny, nz = dims
    r = np.asarray(rho, dtype=np.float64).reshape(nz, ny, nx)
    c = r.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2)
    return c.mean(axis=(1, 3, 5)).reshape(-1)


def transfer(dims_fine, fixed_fine, fixed_coarse) -> sp.csr_matrix:
    """P~ = diag(free_fine) P diag(free_coarse)."""
    P = prolongation_dofs(coarse_dims(dims_fine))
    ff = sp.diags(1.0 - np.asarray(fixed_fine, dtype=np.float64))
    fc = sp.diags(1.0 - np.asarray(fixed_coarse, dtype=np.float64))
    return (ff @ P @ fc).tocsr()


@dataclass
class Level:
    dims: tuple
    K: sp.csr_matrix          # operator with Dirichlet identity rows
    Dinv: np.ndarray          # 1 / diag(K)
    fixed: np.ndarray
    P: sp.csr_matrix | None   # from the next coarser level to this one
    rho: np.ndarray | None = None
    E: np.ndarray | None = None


def homogenized_hierarchy(dims, rho, fixed, K0, levels, E0=1.0, Emin=1e-9, penal=3.0, rule="density"):
    """Levels 0..levels-1 with rediscretised coarse operators.  rule="density"
    (the paper's): coarse E = SIMP(mean of the children's densities);
    rule="modulus" (a variant): coarse E = mean of the children's E."""
    out = []
    d, r, fx = tuple(dims), np.asarray(rho, dtype=np.float64), np.asarray(fixed, dtype=np.uint8)
    E = simp_modulus(r, E0, Emin, penal)
    for l in range(levels):
        if rule == "density" or l == 0:
            E = simp_modulus(r, E0, Emin, penal)
        K = apply_dirichlet(assemble(d, E, (2.0 ** l) * K0), fx)
        out.append(Level(d, K, 1.0 / K.diagonal(), fx, None, r, E))
        if l + 1 < levels:
            fxc = inject_fixed(d, fx)
            out[-1].P = transfer(d, fx, fxc)
            E = homogenize_density(E, d)
            r = homogenize_density(r, d)
            d = coarse_dims(d)
            fx = fxc
    return out


def galerkin_hierarchy(dims, K_fine, fixed, levels):
    """Levels with Galerkin coarse operators K_{l+1} = P~^T K_l P~ (+ identity
    on coarse fixed DOFs), the stored-operator variant of Sec. 4.2.2."""
    out = []
    d, K, fx = tuple(dims), K_fine, np.asarray(fixed, dtype=np.uint8)
    for l in range(levels):
        out.append(Level(d, K, 1.0 / K.diagonal(), fx, None))
        if l + 1 < levels:
            fxc = inject_fixed(d, fx)
            P = transfer(d, fx, fxc)
            out[-1].P = P
            Kc = (P.T @ K @ P).tocsr() + sp.diags(fxc.astype(np.float64))
            d, K, fx = coarse_dims(d), Kc.tocsr(), fxc
    return out


def jacobi(level: Level, u, f, omega):
    return u + omega * level.Dinv * (f - level.K @ u)


def vcycle(levels, f, omega=0.35, pre=2, post=2, l=0, coarse_solve=None):
    """Algorithm 3: one V-cycle from a zero initial iterate, returns u ~ K^-1 f."""
    lev = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(f) if coarse_solve is not None else solve_dense(lev.K, f)
    u = np.zeros_like(f)
    for _ in range(pre):
        u = jacobi(lev, u, f, omega)
    r = f - lev.K @ u
    rc = lev.P.T @ r
    ec = vcycle(levels, rc, omega, pre, post, l + 1, coarse_solve)
    u = u + lev.P @ ec
    for _ in range(post):
        u = jacobi(lev, u, f, omega)
    return u


def max_levels(dims, coarsest_dofs=2500):
    """Number of levels until the coarsest grid has <= coarsest_dofs DOFs."""
    L = 1
    d = tuple(dims)
    while all(x % 2 == 0 for x in d) and 3 * (d[0] + 1) * (d[1] + 1) * (d[2] + 1) > coarsest_dofs:
        d = coarse_dims(d)
        L += 1
    return L


def mgpcg_galerkin(K, f, dims, fixed, tol=1e-12, max_it=2000, levels=None, x0=None,
                   omega=0.35, pre=2, post=2):
    """PCG preconditioned by a Galerkin-operator V-cycle.  Returns (u, it, relres)."""
    L = levels or max_levels(dims)
    hier = galerkin_hierarchy(dims, K, fixed, L)
    Lc = np.linalg.cholesky(hier[-1].K.toarray())

    def coarse(b):
        import scipy.linalg as sla
        y = sla.solve_triangular(Lc, b, lower=True)
        return sla.solve_triangular(Lc.T, y, lower=False)

    return pcg(K, f, lambda r: vcycle(hier, r, omega, pre, post, 0, coarse), tol, max_it, x0)
