"""The host-buffer state step (topo_state_step_host) against the device-pointer
calls it stands for and against the oracle.

The host step copies the density in, solves, forms C and dc and copies dc
out; on the same handle, reset to u = 0 before each, it launches the same
kernels on the same inputs as set_density + solve_state +
compliance_and_sensitivity, so C and dc agree exactly.  Against the oracle:
the FP64 bars of the solve tests (C and u_e energies at rel_tol 1e-10:
1e-8 on C, 1e-7 of max |dc| on dc).
"""
import numpy as np
import pytest

import synth
from oracle import filter as oflt, state as ostate
from gpu_common import cuda_device, n, t

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_host_step_matches_device_calls_and_oracle(precision):
    import torch
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_OK
    dims, levels = (24, 12, 12), 3
    pb = synth.cantilever(dims)
    rho = oflt.density_filter(synth.uniform_field(dims, 4, 1e-3, 1.0), dims, 1.5)
    g = TopoGrid(dims, Params(levels=levels, precision=precision))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    # device-pointer path
    g.set_density(t(rho))
    g.reset_solution()
    _, res_d = g.solve(1e-10, 500)
    dc_d = torch.empty(g.ne, dtype=torch.float64, device=cuda_device())
    C_d, _ = g.compliance_and_sensitivity(dc_d)
    # host-buffer path, twice (the second call reuses the handle's buffers)
    rho_h = torch.tensor(rho).pin_memory()
    for _ in range(2):
        g.reset_solution()
        dc_h = torch.full((g.ne,), np.nan, dtype=torch.float64).pin_memory()
        C_h, _, res_h = g.state_step_host(rho_h, 1e-10, 500, dc=dc_h)
        assert res_h.status == TOPO_OK and res_h.iters == res_d.iters
        assert C_h == C_d
        assert np.array_equal(dc_h.numpy(), n(dc_d))
    # pageable host memory, no dc copy
    g.reset_solution()
    C_p, dc_none, _ = g.state_step_host(torch.tensor(rho), 1e-10, 500)
    assert dc_none is None and C_p == C_d
    # the oracle
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    C_o, _, dc_o = ostate.compliance_and_sensitivity(dims, rho, u_o, pb.f)
    c_bar, dc_bar = (1e-8, 1e-7) if precision == 0 else (1e-7, 1e-5)
    assert abs(C_h - C_o) <= c_bar * abs(C_o)
    assert np.abs(dc_h.numpy() - dc_o).max() <= dc_bar * np.abs(dc_o).max()
    g.close()


def test_host_step_rejects_bad_arguments():
    import torch
    from paper_2201_12931_gb300 import Params, TopoGrid
    from paper_2201_12931_gb300 import _lib as L
    dims = (8, 4, 4)
    g = TopoGrid(dims, Params(levels=2))
    rho = torch.full((g.ne,), 0.5, dtype=torch.float64)
    with pytest.raises(Exception):            # boundary conditions not set
        g.state_step_host(rho, 1e-8, 100)
    with pytest.raises(TypeError):            # a CUDA tensor is not a host buffer
        g.state_step_host(rho.to(cuda_device()), 1e-8, 100)
    assert g.lib.topo_state_step_host(g._h, None, 1e-8, 100, None, None, None, None) == L.TOPO_BADARG
    g.close()
