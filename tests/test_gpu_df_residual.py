"""GPU parity of the double-FP32 operator kernels (TOPO_DF32) against the
oracle, through the C-ABI.

The kernel reads FP64 u, f and moduli, splits each into two FP32 numbers
and evaluates the modal operator with error-free sums and products, so each
arithmetic step carries a relative error of about 2^-47 of the magnitudes
entering it.  Along the ~12 steps between an input and an output that is
below ~1e-13 of the largest element term, so on random inputs (no
cancellation) the bar is the FP64 kernels' 1e-12 relative to the max norm
of the oracle result.  At a converged solution the residual is many orders
smaller than the terms it is made of; there the bar is stated relative to
the load, 2e-12 ||f||_inf, and the FP64 kernel's own error on the same input
is printed beside it.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import assemble, element, state as ostate
from gpu_common import cuda_device, make_case, n, rel_max, t

pytestmark = pytest.mark.gpu

DF32 = 3
CASES = [((6, 4, 4), 2), ((10, 6, 4), 2), ((13, 7, 5), 1), ((48, 24, 24), 3), ((40, 24, 16), 4)]


@pytest.mark.parametrize("dims,levels", CASES)
def test_df_operator_and_residual_all_levels(dims, levels):
    g, pb, rho, H = make_case(dims, levels, seed=5)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 200 + l, -1.0, 1.0)
        f = synth.uniform_field((nl, 1, 1), 300 + l, -1.0, 1.0)
        f[H[l].fixed.astype(bool)] = 0.0
        y = n(g.apply_operator(t(u), level=l, precision=DF32))
        assert rel_max(y, H[l].K @ u) < 1e-12, (l, rel_max(y, H[l].K @ u))
        r = n(g.residual(t(u), t(f), level=l, precision=DF32))
        assert rel_max(r, f - H[l].K @ u) < 1e-12, (l, rel_max(r, f - H[l].K @ u))


@pytest.mark.parametrize("problem", ["cantilever", "mbb"])
def test_df_residual_at_a_converged_solution(problem):
    """r = f - K u at the oracle's solution (relative residual 1e-12) of a
    high-contrast problem: |r| is ~1e-13 |f| while the element terms are
    O(|f|) or more."""
    dims = (48, 24, 24)
    g, pb, rho, H = make_case(dims, 3, problem=problem, seed=3)
    E = assemble.simp_modulus(rho)
    K, fb = assemble.constrained_system(dims, E, element.element_stiffness(0.3), pb.fixed, pb.f)
    u = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-12, method="mgpcg")
    r_ref = fb - K @ u
    fmax = np.abs(fb).max()
    r_df = n(g.residual(t(u), t(fb), level=0, precision=DF32))
    r_64 = n(g.residual(t(u), t(fb), level=0, precision=0))
    e_df = np.abs(r_df - r_ref).max() / fmax
    e_64 = np.abs(r_64 - r_ref).max() / fmax
    print(f"\n{problem}: |r_ref|/|f| = {np.abs(r_ref).max() / fmax:.2e}  "
          f"df32 error {e_df:.2e}  fp64 error {e_64:.2e}  max|u| {np.abs(u).max():.3e}")
    assert e_df <= 2e-12


@pytest.mark.parametrize("outer", [0, 1])
def test_mixed_solve_reaches_1e10_with_either_outer_residual(outer):
    """The refinement loop of the mixed mode converges to a true FP64
    residual of 1e-10 with the double-FP32 outer residual as with the FP64
    one; the displacement matches the oracle's solution (to 1e-12)."""
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_MIXED
    dims = (48, 24, 24)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 3, 1e-3, 1.0)
    g = TopoGrid(dims, Params(levels=3, precision=TOPO_MIXED, outer_residual=outer))
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
    _, res = g.solve(1e-10, 5000, out=u)
    assert res.status == 0 and res.relres <= 1e-10, res
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-12, method="mgpcg")
    assert np.linalg.norm(n(u) - u_o) <= 1e-8 * np.linalg.norm(u_o)
    E = assemble.simp_modulus(rho)
    K, fb = assemble.constrained_system(dims, E, element.element_stiffness(0.3), pb.fixed, pb.f)
    assert np.linalg.norm(fb - K @ n(u)) <= 1.2e-10 * np.linalg.norm(fb)   # the reported residual is true
    g.close()


def test_df_rejects_modes_it_does_not_offer():
    from paper_2201_12931_gb300 import TopoError
    g, pb, rho, H = make_case((8, 4, 4), 2)
    u = t(np.zeros(H[0].K.shape[0]))
    with pytest.raises(TopoError):
        g.jacobi_sweep(u, u, level=0, precision=DF32)
    g.close()
