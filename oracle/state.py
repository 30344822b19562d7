"""State solve and one topology-optimisation iteration (oracle; test infrastructure only).

solve_state assembles K(rho~) with Dirichlet rows and solves K u = f with a
direct method on small systems and, above that, with PCG (Algorithm 1)
preconditioned by a Galerkin-operator V-cycle (Algorithm 3 with stored
coarse operators).  The preconditioner only changes the path, not the
converged u, so the oracle's u is independent of the GPU's homogenized
V-cycle.

oc_iteration runs one pass of Algorithm 4's loop body with the density
filter: rho~ = H x, solve, compliance, sensitivity, OC update of x.
"""
from __future__ import annotations

import numpy as np

from .assemble import constrained_system, simp_modulus
from .element import element_stiffness
from .filter import density_filter, sensitivity_filter
from .multigrid import homogenized_hierarchy, max_levels, mgpcg_galerkin, vcycle
from .oc import oc_update, oc_update_unfiltered
from .sensitivity import compliance, element_energy, sensitivity
from .solve import pcg, solve_dense, solve_sparse_direct


def solve_state(dims, rho, fixed, f, nu=0.3, E0=1.0, Emin=1e-9, penal=3.0, tol=1e-12,
                method="auto", x0=None, return_info=False):
    K0 = element_stiffness(nu)
    E = simp_modulus(rho, E0, Emin, penal)
    K, fb = constrained_system(dims, E, K0, fixed, f)
    n = fb.size
    if method == "auto":
        method = "dense" if n <= 3000 else ("direct" if n <= 40000 else "mgpcg")
    info = dict(method=method, iters=0, relres=0.0)
    if method == "dense":
        u = solve_dense(K, fb)
    elif method == "direct":
        u = solve_sparse_direct(K, fb)
    elif method == "mgpcg_homog":
        # PCG with the homogenized V-cycle (cheaper set-up than Galerkin
        # products on large grids; the converged u does not depend on M)
        H = homogenized_hierarchy(dims, rho, fixed, K0, max_levels(dims), E0, Emin, penal)
        Lc = np.linalg.cholesky(H[-1].K.toarray())
        import scipy.linalg as sla

        def coarse(b):
            return sla.solve_triangular(Lc.T, sla.solve_triangular(Lc, b, lower=True), lower=False)

        u, it, rr = pcg(K, fb, lambda r: vcycle(H, r, coarse_solve=coarse), tol, 5000, x0)
        info.update(iters=it, relres=rr)
    else:
        u, it, rr = mgpcg_galerkin(K, fb, dims, fixed, tol=tol, x0=x0)
        info.update(iters=it, relres=rr)
    nf = np.linalg.norm(fb)
    info["relres"] = float(np.linalg.norm(fb - K @ u) / nf) if nf > 0 else 0.0
    return (u, info) if return_info else u


def compliance_and_sensitivity(dims, rho, u, f, nu=0.3, E0=1.0, Emin=1e-9, penal=3.0):
    K0 = element_stiffness(nu)
    se = element_energy(u, dims, K0)
    E = simp_modulus(rho, E0, Emin, penal)
    C_energy = float(np.sum(E * se))
    return compliance(f, u), C_energy, sensitivity(rho, se, E0, Emin, penal)


def oc_iteration(dims, x, fixed, f, r, volfrac, move=0.2, nu=0.3, E0=1.0, Emin=1e-9,
                 penal=3.0, tol=1e-10, x0=None):
    """One loop body of Algorithm 4 with a density filter.
    Returns dict(C, x_new, change, u, rho_phys, dc)."""
    rho = density_filter(x, dims, r)
    u = solve_state(dims, rho, fixed, f, nu, E0, Emin, penal, tol=tol, x0=x0)
    C, _, dc = compliance_and_sensitivity(dims, rho, u, f, nu, E0, Emin, penal)
    xn, ch, lam, steps = oc_update(x, dc, dims, r, volfrac, move)
    return dict(C=C, x_new=xn, change=ch, u=u, rho_phys=rho, dc=dc, lam=lam, steps=steps)


def oc_iteration_sensitivity_filter(dims, x, fixed, f, r, volfrac, move=0.2, gamma=1e-3, nu=0.3, E0=1.0,
                                    Emin=1e-9, penal=3.0, tol=1e-10, x0=None):
    """One loop body of Algorithm 4 as the paper runs it: the design is the
    physical density, the sensitivities go through Eq. sensitivity filter,
    then the OC update.  Returns dict(C, x_new, change, u, dc, dc_filtered)."""
    x = np.asarray(x, dtype=np.float64)
    u = solve_state(dims, x, fixed, f, nu, E0, Emin, penal, tol=tol, x0=x0)
    C, _, dc = compliance_and_sensitivity(dims, x, u, f, nu, E0, Emin, penal)
    dcf = sensitivity_filter(x, dc, dims, r, gamma)
    xn, ch, lam, steps = oc_update_unfiltered(x, dcf, volfrac, move)
    return dict(C=C, x_new=xn, change=ch, u=u, dc=dc, dc_filtered=dcf, lam=lam, steps=steps)
