"""Pins of the oracle's grid transfers, homogenized hierarchy and V-cycle.

* the interpolation reproduces trilinear fields exactly;
* restriction is its transpose (dot-product test);
* Galerkin identity: for uniform stiffness P~^T K_h P~ equals the
  rediscretised coarse operator built from 2 K0 -- this checks the transfer
  weights, the 2^l element scaling, the Dirichlet injection and the density
  averaging of the homogenized hierarchy together;
* the printed 1D restriction stencil (1/4)[1 2 1] (Sec. 4.2.2) is
  proportional to the transpose of interpolation (golden fixture);
* the V-cycle is a symmetric positive definite operator, equals a direct
  solve with one level, and with uniform stiffness and no smoothing its
  two-level error propagator is a K-orthogonal projector.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import assemble, element, grid, multigrid

NU = 0.3
K0 = element.element_stiffness(NU)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_interpolation_reproduces_trilinear_fields():
    dc = (3, 2, 2)
    df = (6, 4, 4)
    P = multigrid.prolongation_nodes(dc)
    Xc = grid.node_coords(dc).astype(float) * 2.0
    Xf = grid.node_coords(df).astype(float)

    def field(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return 1.0 + 0.3 * x - 0.2 * y + 0.5 * z + 0.1 * x * y - 0.07 * y * z + 0.02 * x * z + 0.01 * x * y * z

    assert np.abs(P @ field(Xc) - field(Xf)).max() < 1e-12


def test_restriction_is_transpose():
    dc = (2, 2, 1)
    P = multigrid.prolongation_dofs(dc)
    rng = np.random.default_rng(0)
    a = rng.standard_normal(P.shape[1])
    b = rng.standard_normal(P.shape[0])
    assert (P @ a) @ b == pytest.approx(a @ (P.T @ b), rel=1e-13)


def test_restriction_stencil_matches_printed_rows():
    with open(os.path.join(GOLDEN, "restriction_1d.json")) as fh:
        g = json.load(fh)
    R = multigrid.prolongation_1d(4).T.toarray()
    printed = np.array(g["row"], dtype=float) * g["scale"]
    interior = R[1, 1:4]                       # coarse node 1 <- fine nodes 1, 2, 3
    ratio = interior / printed
    assert np.allclose(ratio, ratio[0])
    assert ratio[0] == pytest.approx(2.0)


@pytest.mark.parametrize("problem", ["cantilever", "mbb"])
def test_galerkin_identity_uniform_density(problem):
    dims = (4, 4, 2) if problem == "cantilever" else (8, 4, 4)
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    rho = np.full(grid.n_elems(dims), 0.7)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=2)
    Kg = (H[0].P.T @ H[0].K @ H[0].P).toarray()
    fixed_c = H[1].fixed.astype(bool)
    Kg[fixed_c, fixed_c] = 1.0
    assert np.abs(Kg - H[1].K.toarray()).max() < 1e-12 * np.abs(Kg).max()


@pytest.mark.parametrize("problem", ["cantilever", "mbb"])
def test_galerkin_hierarchy_equals_rediscretisation_for_uniform_density(problem):
    """Pins galerkin_hierarchy (assembled P~^T K P~) against the independent
    rediscretisation with 2^l K0 on three levels: they coincide for uniform
    stiffness."""
    dims = (8, 8, 4) if problem == "cantilever" else (8, 4, 4)
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    rho = np.full(grid.n_elems(dims), 0.6)
    Hh = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=3)
    Hg = multigrid.galerkin_hierarchy(dims, Hh[0].K, pb.fixed, levels=3)
    for a, b in zip(Hg, Hh):
        assert np.abs((a.K - b.K).toarray()).max() < 1e-12 * np.abs(b.K.toarray()).max()


def test_homogenized_density_is_child_mean():
    dims = (4, 2, 2)
    rho = synth.uniform_field(dims, 11)
    rc = multigrid.homogenize_density(rho, dims)
    r3 = rho.reshape(2, 2, 4)
    assert rc.shape == (2,)
    assert rc[0] == pytest.approx(r3[:, :, 0:2].mean())
    assert rc[1] == pytest.approx(r3[:, :, 2:4].mean())


def test_homogenized_operator_is_not_galerkin_for_varying_density():
    """The homogenized coarse operator is a rediscretisation, not P^T K P."""
    dims = (4, 4, 4)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 5, 0.1, 1.0)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=2)
    Kg = (H[0].P.T @ H[0].K @ H[0].P).toarray()
    fc = H[1].fixed.astype(bool)
    Kg[fc, fc] = 1.0
    assert np.abs(Kg - H[1].K.toarray()).max() > 1e-3 * np.abs(Kg).max()


def _linear_field(dims, A, h=1.0):
    """Nodal values of u(x) = A x on a grid of element size h (node-major)."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = h * np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    return (X @ A.T).reshape(-1)


@pytest.mark.parametrize("levels", [2, 3])
def test_modulus_rule_reproduces_linear_field_energy(levels):
    """Averaging the moduli gives each coarse element the energy its 8^l fine
    descendants store under any uniform strain (a linear displacement field
    has the same strain in every child), so u_c^T K_c u_c = u_f^T K_h u_f.
    Averaging the densities instead stores less (Jensen: mean(rho)^3 <=
    mean(rho^3)).  Pins the modulus averaging, the 2^l element scaling and
    their chaining over levels."""
    dims = (8, 8, 4)
    rho = synth.uniform_field(dims, 21, 0.0, 1.0)
    free = np.zeros(3 * grid.n_nodes(dims), dtype=np.uint8)
    A = synth.uniform_field((3, 3, 1), 22, -1.0, 1.0).reshape(3, 3)
    Hm = multigrid.homogenized_hierarchy(dims, rho, free, K0, levels, rule="modulus")
    Hd = multigrid.homogenized_hierarchy(dims, rho, free, K0, levels, rule="density")
    uf = _linear_field(dims, A)
    ef = uf @ (Hm[0].K @ uf)
    for l in range(1, levels):
        uc = _linear_field(Hm[l].dims, A, h=2.0 ** l)
        assert uc @ (Hm[l].K @ uc) == pytest.approx(ef, rel=1e-12)
        assert uc @ (Hd[l].K @ uc) < 0.9 * ef


def test_modulus_rule_equals_density_rule_for_uniform_density():
    dims = (8, 4, 4)
    pb = synth.cantilever(dims)
    rho = np.full(grid.n_elems(dims), 0.37)
    Hm = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, 3, rule="modulus")
    Hd = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, 3, rule="density")
    for a, b in zip(Hm, Hd):
        assert np.abs((a.K - b.K).toarray()).max() < 1e-14 * np.abs(b.K.toarray()).max()


def _vcycle_matrix(H, **kw):
    n = H[0].K.shape[0]
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = multigrid.vcycle(H, e, **kw)
    return M


def test_jacobi_bound_theta():
    """lambda_max(D^-1 K) <= lambda_max(diag(K0)^-1 K0) = theta for any density."""
    d = np.sqrt(np.diag(K0))
    theta = np.linalg.eigvalsh(K0 / np.outer(d, d))[-1]
    assert 2.0 / theta > 0.35
    dims = (4, 4, 2)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 3, 1e-3, 1.0)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=1)
    K = H[0].K.toarray()
    s = np.sqrt(np.diag(K))
    assert np.linalg.eigvalsh(K / np.outer(s, s))[-1] <= theta + 1e-12


def test_vcycle_symmetric_positive_definite():
    dims = (4, 4, 4)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 9, 1e-3, 1.0)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=3)
    M = _vcycle_matrix(H, omega=0.35, pre=2, post=2)
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T))[0] > 0


def test_vcycle_indefinite_with_large_damping():
    """omega = 0.6 exceeds 2/theta: on a high-contrast field the V-cycle loses
    positive definiteness, which is why the default damping is 0.35."""
    dims = (4, 4, 4)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 9, 1e-3, 1.0)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=3)
    M = _vcycle_matrix(H, omega=0.6, pre=2, post=2)
    assert np.linalg.eigvalsh(0.5 * (M + M.T))[0] < 0


def test_vcycle_one_level_is_direct_solve():
    dims = (2, 2, 2)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 4, 0.2, 1.0)
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels=1)
    f = np.where(pb.fixed.astype(bool), 0.0, synth.uniform01(8, pb.f.size))
    u = multigrid.vcycle(H, f)
    assert np.abs(H[0].K @ u - f).max() < 1e-12


def test_two_level_coarse_correction_is_k_projector():
    dims = (4, 4, 4)
    pb = synth.cantilever(dims)
    H = multigrid.homogenized_hierarchy(dims, np.full(64, 0.5), pb.fixed, K0, levels=2)
    M = _vcycle_matrix(H, pre=0, post=0)
    K = H[0].K.toarray()
    T = np.eye(K.shape[0]) - M @ K
    assert np.abs(T @ T - T).max() < 1e-9
    assert np.abs(K @ T - (K @ T).T).max() < 1e-9 * np.abs(K).max()


def test_coarse_dirichlet_injection():
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    fc = multigrid.inject_fixed(dims, pb.fixed).reshape(-1, 3)
    Xc = grid.node_coords((2, 1, 1))
    assert np.all(fc[Xc[:, 0] == 0] == 1)
    assert np.all(fc[Xc[:, 0] > 0] == 0)
