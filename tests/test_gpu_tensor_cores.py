"""GPU parity of the FP32 operator kernels with tensor-core element products
(TOPO_FP32_TC, topo_params.tensor_cores = 1) against the oracle, through the
C-ABI.

The element products K0 (u_e - u_e0) run on the tcgen05 tensor cores with
TF32 operands split into hi + lo (hi K0_hi + hi K0_lo + lo K0_hi, FP32
accumulation): each product carries about 2^-22 of relative error, against
2^-24 for the modal CUDA-core kernel, and the sums over 24 terms stay well
inside the FP32 kernels' bars: 1e-5 (K.u, residual) and 2e-5 (Jacobi sweep)
relative to the max norm of the oracle result.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import multigrid, state as ostate, filter as oflt
from gpu_common import cuda_device, make_case, n, rel_max, t

pytestmark = pytest.mark.gpu

TC = 4
CASES = [((6, 4, 4), 2), ((10, 6, 4), 2), ((13, 7, 5), 1), ((48, 24, 24), 3), ((40, 24, 16), 4), ((70, 20, 36), 2)]


@pytest.mark.parametrize("dims,levels", CASES)
def test_tc_operator_jacobi_residual_all_levels(dims, levels):
    g, pb, rho, H = make_case(dims, levels, seed=6)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 400 + l, -1.0, 1.0)
        f = synth.uniform_field((nl, 1, 1), 500 + l, -1.0, 1.0)
        f[H[l].fixed.astype(bool)] = 0.0
        y = n(g.apply_operator(t(u), level=l, precision=TC))
        assert rel_max(y, H[l].K @ u) < 1e-5, (l, rel_max(y, H[l].K @ u))
        uj = n(g.jacobi_sweep(t(u), t(f), level=l, precision=TC))
        ref = multigrid.jacobi(H[l], u, f, g.params.omega)
        assert rel_max(uj, ref) < 2e-5, (l, rel_max(uj, ref))
        r = n(g.residual(t(u), t(f), level=l, precision=TC))
        assert rel_max(r, f - H[l].K @ u) < 1e-5, (l, rel_max(r, f - H[l].K @ u))


def test_tc_operator_on_a_smooth_field():
    """A displacement that is nearly a rigid translation at element scale
    (smooth, large mean): the corner-0 shift keeps the result accurate."""
    dims, levels = (48, 24, 24), 3
    g, pb, rho, H = make_case(dims, levels, seed=3)
    nn = H[0].K.shape[0] // 3
    k, j, i = np.meshgrid(np.arange(dims[2] + 1), np.arange(dims[1] + 1), np.arange(dims[0] + 1), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(float)
    u = (100.0 + np.sin(X / 7.0) + 0.01 * X ** 2 / 48.0).ravel()
    y = n(g.apply_operator(t(u), level=0, precision=TC))
    assert rel_max(y, H[0].K @ u) < 1e-5, rel_max(y, H[0].K @ u)


@pytest.mark.parametrize("dims,levels,problem", [((48, 24, 24), 3, "cantilever"), ((32, 16, 16), 4, "mbb")])
def test_mixed_solve_with_tensor_cores_matches_oracle(dims, levels, problem):
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_MIXED
    rho = oflt.density_filter(synth.uniform_field(dims, 1, 1e-3, 1.0), dims, 1.5)
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    g = TopoGrid(dims, Params(levels=levels, precision=TOPO_MIXED, tensor_cores=1))
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
    _, res = g.solve(1e-8, 5000, out=u)
    assert res.status == 0 and res.relres <= 1e-8, res
    assert np.linalg.norm(n(u) - u_o) <= 1e-6 * np.linalg.norm(u_o)
    g.close()
