"""Planted mistakes: each pin must catch a plausible error in the oracle.

Every case builds a mutated copy of one oracle function on the CPU and
checks that the corresponding pin, which passes for the real oracle, fails
for the mutant.  Nothing here touches the CUDA path.
"""
import numpy as np
import scipy.sparse as sp

import synth
from oracle import assemble, element, filter as flt, grid, multigrid, sensitivity, solve


def _patch_residual(K0):
    dims = (3, 3, 3)
    K = assemble.assemble(dims, np.ones(27), K0)
    X = grid.node_coords(dims).astype(float)
    u = (X @ np.array([[0.2, -0.1, 0.3], [0.4, 0.1, -0.2], [-0.3, 0.2, 0.05]]).T).ravel()
    y = (K @ u).reshape(-1, 3)
    inner = np.all((X > 0) & (X < 3), axis=1)
    return np.abs(y[inner]).max()


def test_real_k0_passes_patch():
    assert _patch_residual(element.element_stiffness(0.3)) < 1e-13


def test_wrong_shear_sign_is_caught():
    def bad(nu=0.3):
        D = element.elasticity_matrix(1.0, nu)
        D[3:, 3:] *= -1.0
        xg, wg = np.polynomial.legendre.leggauss(2)
        K = np.zeros((24, 24))
        for i in range(2):
            for j in range(2):
                for k in range(2):
                    B = element.strain_displacement(0.5 * (xg[i] + 1), 0.5 * (xg[j] + 1), 0.5 * (xg[k] + 1))
                    K += 0.125 * wg[i] * wg[j] * wg[k] * (B.T @ D @ B)
        return K
    Kb = bad()
    Kx = np.array([[float(v) for v in row] for row in element.element_stiffness_exact()])
    assert np.abs(Kb - Kx).max() > 1e-3
    assert np.linalg.eigvalsh(Kb)[0] < -1e-3


def _uniform_strain_energy_error(K0):
    lam, mu = element.lame(1.0, 0.3)
    A = np.array([[0.3, 0.1, -0.2], [0.05, -0.4, 0.2], [0.1, 0.25, 0.15]])
    u = np.concatenate([A @ np.array(c, dtype=float) for c in element.CORNERS])
    eps = 0.5 * (A + A.T)
    return abs(u @ K0 @ u - (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)))


def test_swapped_corner_order_is_caught():
    """A relabelled K0 keeps zero row sums, so the interior patch test alone
    misses it; the uniform-strain energy pin catches it."""
    K0 = element.element_stiffness(0.3)
    assert _uniform_strain_energy_error(K0) < 1e-14
    for perm in ([0, 1, 3, 2, 4, 5, 6, 7], [1, 0, 2, 3, 4, 5, 6, 7]):
        dof = np.array([3 * a + c for a in perm for c in range(3)])
        assert _uniform_strain_energy_error(K0[np.ix_(dof, dof)]) > 1e-3


def test_swapped_components_are_caught():
    K0 = element.element_stiffness(0.3)
    dof = np.array([3 * a + c for a in range(8) for c in (1, 0, 2)])
    assert _uniform_strain_energy_error(K0[np.ix_(dof, dof)]) > 1e-3


def test_quarter_restriction_breaks_galerkin_identity():
    dims, dc = (4, 2, 2), (2, 1, 1)
    K0 = element.element_stiffness(0.3)
    Kf = assemble.assemble(dims, np.ones(16), K0)
    Kc = assemble.assemble(dc, np.ones(2), 2 * K0).toarray()
    P = multigrid.prolongation_dofs(dc)
    good = np.abs((P.T @ Kf @ P).toarray() - Kc).max()
    bad = np.abs((0.5 * P.T @ Kf @ P).toarray() - Kc).max()   # rows (1/4)[1 2 1]
    assert good < 1e-13 and bad > 1e-2


def test_unscaled_coarse_element_breaks_galerkin_identity():
    dims, dc = (4, 2, 2), (2, 1, 1)
    K0 = element.element_stiffness(0.3)
    Kf = assemble.assemble(dims, np.ones(16), K0)
    P = multigrid.prolongation_dofs(dc)
    Kc_bad = assemble.assemble(dc, np.ones(2), K0).toarray()   # missing 2^l
    assert np.abs((P.T @ Kf @ P).toarray() - Kc_bad).max() > 1e-2


def test_unnormalised_filter_is_caught():
    dims = (5, 4, 3)
    x = np.full(60, 0.5)
    acc = np.zeros((3, 4, 5))
    for dx, dy, dz, w in flt.offsets(1.5):
        flt._shift_accumulate(acc, x.reshape(3, 4, 5), dx, dy, dz, w)
    bad = acc.ravel() / flt.weight_sums(dims, 1.5).max()     # global instead of local S_e
    assert np.abs(bad - 0.5).max() > 1e-3


def test_transpose_without_normalisation_is_caught():
    dims = (6, 5, 4)
    a = synth.uniform_field(dims, 1)
    b = synth.uniform_field(dims, 2, -1.0, 1.0)
    acc = np.zeros((4, 5, 6))
    for dx, dy, dz, w in flt.offsets(2.0):
        flt._shift_accumulate(acc, b.reshape(4, 5, 6), dx, dy, dz, w)
    bad_T = acc.ravel() / flt.weight_sums(dims, 2.0)         # divides after summing
    lhs = flt.density_filter(a, dims, 2.0) @ b
    assert abs(lhs - a @ bad_T) > 1e-6 * abs(lhs)


def test_sensitivity_missing_exponent_is_caught():
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 13, 0.2, 1.0)
    K0 = element.element_stiffness(0.3)
    E = assemble.simp_modulus(rho)
    K, fb = assemble.constrained_system(dims, E, K0, pb.fixed, pb.f)
    u = solve.solve_dense(K, fb)
    se = sensitivity.element_energy(u, dims, K0)
    bad = -3.0 * rho ** 3 * se                                # p rho^p instead of p rho^(p-1)
    h = 1e-5
    rp, rm = rho.copy(), rho.copy()
    rp[3] += h
    rm[3] -= h

    def C(r):
        Kr, fr = assemble.constrained_system(dims, assemble.simp_modulus(r), K0, pb.fixed, pb.f)
        return fr @ solve.solve_dense(Kr, fr)

    fd = (C(rp) - C(rm)) / (2 * h)
    assert abs(bad[3] - fd) > 1e-2 * abs(fd)


def test_dropped_dirichlet_column_is_caught():
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    K0 = element.element_stiffness(0.3)
    K = assemble.assemble(dims, np.ones(16), K0)
    fixed = pb.fixed.astype(bool)
    bad = sp.lil_matrix(K)
    bad[np.where(fixed)[0], :] = 0.0                          # rows only, columns kept
    bad = bad.tocsr() + sp.diags(fixed.astype(float))
    assert np.abs((bad - bad.T).toarray()).max() > 1e-3


# ---- planted mistakes in the added oracle functions -------------------------

def test_sensitivity_filter_without_gamma_clamp_is_caught():
    """Dividing by rho_e instead of max(gamma, rho_e): the brute-force pin with
    densities below gamma fails."""
    dims = (5, 4, 3)
    rho = synth.uniform_field(dims, 31, 0.0, 1.0)
    rho[::7] = 1e-4
    dc = -synth.uniform_field(dims, 32, 0.1, 5.0)
    ref = flt.density_filter_bruteforce(rho * dc, dims, 1.5) / np.maximum(1e-3, rho)
    bad = flt.density_filter(rho * dc, dims, 1.5) / rho
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


def test_gravity_term_with_wrong_factor_is_caught():
    """u_e^T g_e instead of 2 u_e^T g_e: central differences disagree."""
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    K0 = element.element_stiffness(0.3)
    rho = synth.uniform_field(dims, 7, 0.3, 1.0)
    w = 0.7

    def solve_c(r):
        f = sensitivity.gravity_load(dims, r, w, pb.f)
        K, fb = assemble.constrained_system(dims, assemble.simp_modulus(r), K0, pb.fixed, f)
        u = np.linalg.solve(K.toarray(), fb)
        return float(fb @ u), u

    _, u = solve_c(rho)
    se = sensitivity.element_energy(u, dims, K0)
    bad = sensitivity.sensitivity(rho, se) + 0.5 * sensitivity.gravity_sensitivity_term(dims, u, w)
    e, h = 3, 1e-6
    rp, rm = rho.copy(), rho.copy()
    rp[e] += h
    rm[e] -= h
    fd = (solve_c(rp)[0] - solve_c(rm)[0]) / (2 * h)
    assert abs(bad[e] - fd) > 1e-4 * abs(fd)


def test_modulus_rule_without_element_scale_is_caught():
    """Averaging the moduli but dropping the factor 2 per level: the coarse
    energy of a linear field no longer matches the fine one."""
    dims = (8, 8, 4)
    rho = synth.uniform_field(dims, 21, 0.0, 1.0)
    K0 = element.element_stiffness(0.3)
    E = assemble.simp_modulus(rho)
    Kf = assemble.assemble(dims, E, K0)
    Ec = multigrid.homogenize_density(E, dims)
    Kc_bad = assemble.assemble(multigrid.coarse_dims(dims), Ec, K0)          # missing 2 K0
    A = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, 0.25]])

    def lin(d, h):
        nx, ny, nz = d
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        X = h * np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(float)
        return (X @ A.T).ravel()
    uf, uc = lin(dims, 1.0), lin(multigrid.coarse_dims(dims), 2.0)
    assert abs(uc @ (Kc_bad @ uc) - uf @ (Kf @ uf)) > 0.3 * abs(uf @ (Kf @ uf))


def test_passive_volume_over_all_elements_is_caught():
    """Bisecting on the volume of all elements instead of the active ones:
    the active volume fraction misses the target."""
    from oracle import oc
    x = np.full(128, 0.3)
    passive = np.zeros(128, dtype=np.uint8)
    passive[:16] = 1
    x[:16] = 1.0
    dc = -synth.uniform_field((8, 4, 4), 3, 0.1, 10.0)
    bad = oc.oc_update_unfiltered(x, dc, 0.3, 0.2)[0]        # passive ignored
    bad[:16] = 1.0
    good = oc.oc_update_unfiltered(x, dc, 0.3, 0.2, passive=passive)[0]
    assert abs(good[16:].mean() - 0.3) < 1e-6
    assert abs(bad[16:].mean() - 0.3) > 1e-2


def _oc_with_law(law, use_dv=True):
    """Mutated copy of oracle.oc.oc_update whose unclamped candidate is
    law(x, B) instead of x B^(1/2); use_dv=False drops the filter transpose
    of the volume derivative (dv~ = 1)."""
    def update(x, dc, dims, r, volfrac, move):
        dct = flt.density_filter_T(dc, dims, r)
        dvt = flt.density_filter_T(np.ones_like(x), dims, r) if use_dv else np.ones_like(x)
        num = np.maximum(-dct, 1e-30)
        l1, l2 = 0.0, 1e9
        xnew = x.copy()
        while (l2 - l1) / (l1 + l2) > 1e-9:
            lmid = 0.5 * (l1 + l2)
            cand = law(x, num / (lmid * dvt))
            xnew = np.maximum(0.0, np.maximum(x - move, np.minimum(1.0, np.minimum(x + move, cand))))
            if flt.density_filter(xnew, dims, r).mean() > volfrac:
                l1 = lmid
            else:
                l2 = lmid
        return xnew, None
    return update


def test_oc_law_mistakes_are_caught():
    """eta = 1, the paper's q = 2 on the unclamped value, and a volume
    derivative without the filter transpose each leave the minimiser of the
    reciprocal-variable subproblem (the pin in test_oracle_oc_law.py);
    the law as read (eta = 1/2, q = 1) passes through the same copy."""
    from test_oracle_oc_law import _filtered_case, oc_law_error
    case = _filtered_case()
    assert oc_law_error(_oc_with_law(lambda x, B: x * np.sqrt(B)), *case)[0] < 1e-6
    for bad in (_oc_with_law(lambda x, B: x * B),
                _oc_with_law(lambda x, B: (x * np.sqrt(B)) ** 2),
                _oc_with_law(lambda x, B: x * np.sqrt(B), use_dv=False)):
        assert oc_law_error(bad, *case)[0] > 1e-3
