"""Pins of the oracle's assembled operator and state solve.

Closed forms: patch test (linear fields give zero interior forces), the
uniaxial bar (exact u and C = sigma^2 V / E), the energy identity, PCG
against a library dense solve, and agreement of three solve routes.
"""
import numpy as np
import pytest

import synth
from oracle import assemble, element, grid, multigrid, solve, state
from oracle.sensitivity import element_energy

NU = 0.3


def test_patch_test_interior_forces_vanish():
    dims = (4, 3, 3)
    K = assemble.assemble(dims, np.ones(grid.n_elems(dims)), element.element_stiffness(NU))
    X = grid.node_coords(dims).astype(float)
    A = np.array([[0.2, -0.1, 0.3], [0.4, 0.1, -0.2], [-0.3, 0.2, 0.05]])
    b = np.array([0.7, -0.2, 0.1])
    u = (X @ A.T + b).ravel()
    y = (K @ u).reshape(-1, 3)
    nx, ny, nz = dims
    inner = (X[:, 0] > 0) & (X[:, 0] < nx) & (X[:, 1] > 0) & (X[:, 1] < ny) & (X[:, 2] > 0) & (X[:, 2] < nz)
    assert np.abs(y[inner]).max() < 1e-13
    assert np.abs(y[~inner]).max() > 1e-3      # boundary tractions are not zero


def _bar(dims, E=1.0, sigma=1.0):
    nx, ny, nz = dims
    X = grid.node_coords(dims)
    fixed = np.zeros((X.shape[0], 3), dtype=np.uint8)
    fixed[X[:, 0] == 0, 0] = 1
    fixed[X[:, 1] == 0, 1] = 1
    fixed[X[:, 2] == 0, 2] = 1
    f = np.zeros((X.shape[0], 3))
    # consistent nodal forces of a uniform traction on the face x = nx
    wy = np.where((X[:, 1] == 0) | (X[:, 1] == ny), 0.5, 1.0)
    wz = np.where((X[:, 2] == 0) | (X[:, 2] == nz), 0.5, 1.0)
    f[:, 0] = np.where(X[:, 0] == nx, sigma * wy * wz, 0.0)
    return X, fixed.ravel(), f.ravel()


@pytest.mark.parametrize("dims", [(3, 2, 2), (6, 3, 2)])
def test_uniaxial_bar_exact_solution(dims):
    E, sigma = 1.0, 0.8
    X, fixed, f = _bar(dims, E, sigma)
    rho = np.ones(grid.n_elems(dims))
    u = state.solve_state(dims, rho, fixed, f, nu=NU, Emin=0.0, method="dense")
    exact = np.stack([sigma * X[:, 0] / E, -NU * sigma * X[:, 1] / E, -NU * sigma * X[:, 2] / E], 1).ravel()
    assert np.abs(u - exact).max() < 1e-12
    V = float(np.prod(dims))
    assert f @ u == pytest.approx(sigma ** 2 * V / E, rel=1e-12)


def test_energy_identity_and_three_solvers():
    dims = (6, 4, 4)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 7, 0.05, 1.0)
    K0 = element.element_stiffness(NU)
    E = assemble.simp_modulus(rho)
    K, fb = assemble.constrained_system(dims, E, K0, pb.fixed, pb.f)
    u1 = solve.solve_dense(K, fb)
    u2 = solve.solve_sparse_direct(K, fb)
    u3, it, rr = multigrid.mgpcg_galerkin(K, fb, dims, pb.fixed, tol=1e-13, levels=2)
    assert rr <= 1e-13
    for u in (u2, u3):
        assert np.linalg.norm(u - u1) <= 1e-9 * np.linalg.norm(u1)
    C = fb @ u1
    assert u1 @ (K @ u1) == pytest.approx(C, rel=1e-12)
    assert np.sum(E * element_energy(u1, dims, K0)) == pytest.approx(C, rel=1e-12)
    assert np.all(u1[pb.fixed.astype(bool)] == 0.0)


def test_pcg_against_library_solve():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 60))
    A = A @ A.T + 60 * np.eye(60)
    b = rng.standard_normal(60)
    d = np.diag(A)
    x, it, rr = solve.pcg(A, b, lambda r: r / d, tol=1e-13)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-10
    assert it < 60


def test_mbb_constraints_remove_rigid_motion():
    dims = (4, 2, 2)
    pb = synth.mbb_half(dims)
    K, _ = assemble.constrained_system(dims, np.ones(16), element.element_stiffness(NU), pb.fixed, pb.f)
    ev = np.linalg.eigvalsh(K.toarray())
    assert ev[0] > 1e-6


def test_cantilever_deflects_down_and_grows_with_softness():
    dims = (8, 4, 4)
    pb = synth.cantilever(dims)
    u1 = state.solve_state(dims, np.full(128, 1.0), pb.fixed, pb.f, method="direct")
    u2 = state.solve_state(dims, np.full(128, 0.5), pb.fixed, pb.f, method="direct")
    tip = 3 * int(synth.node_index(dims, 8, 2, 0)) + 2
    assert u1[tip] < 0
    # uniform rho scales E by rho^3 (Emin negligible): u scales by 1/rho^3
    assert u2[tip] == pytest.approx(8.0 * u1[tip], rel=1e-6)


def test_gravity_load_resultant():
    from oracle import sensitivity as osens
    dims = (4, 3, 2)
    rho = synth.uniform_field(dims, 9, 0.1, 1.0)
    f = osens.gravity_load(dims, rho, 2.5)
    assert f[2::3].sum() == pytest.approx(-2.5 * rho.sum(), rel=1e-14)
    assert np.all(f[0::3] == 0.0) and np.all(f[1::3] == 0.0)


def test_gravity_sensitivity_central_differences():
    """C(rho) = f(rho)^T u(rho) with the self-weight load, dense direct solves:
    the adjoint gradient 2 u^T df/drho - u^T dK/drho u against central
    differences on every element of a tiny grid."""
    from oracle import assemble as oas, element as oel, sensitivity as osens
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    K0 = oel.element_stiffness(0.3)
    rho = synth.uniform_field(dims, 7, 0.3, 1.0)
    w = 0.7

    def solve(r):
        f = osens.gravity_load(dims, r, w, pb.f)
        K, fb = oas.constrained_system(dims, oas.simp_modulus(r), K0, pb.fixed, f)
        u = np.linalg.solve(K.toarray(), fb)
        return float(fb @ u), u

    C, u = solve(rho)
    g = osens.sensitivity(rho, osens.element_energy(u, dims, K0)) + osens.gravity_sensitivity_term(dims, u, w)
    h = 1e-6
    for e in range(rho.size):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (solve(rp)[0] - solve(rm)[0]) / (2 * h)
        assert fd == pytest.approx(g[e], rel=1e-6, abs=1e-9 * abs(C))
