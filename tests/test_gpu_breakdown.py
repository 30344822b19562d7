"""The solver's failure contract on singular problems made on the host
(no GPU fault is involved): Dirichlet conditions that leave rigid-body modes
free make K singular.  topo_solve_state must return TOPO_BREAKDOWN or
TOPO_MAXITER with a finite best iterate and its FP64 residual, a message in
topo_last_error, and the handle must solve the well-posed problem afterwards.
Every loop of the solver is bounded (max_it, refinement steps, restarts).
"""
import numpy as np
import pytest
import torch

import synth
from gpu_common import cuda_device, n, t

pytestmark = pytest.mark.gpu


def _singular_masks(dims):
    pb = synth.cantilever(dims)
    free = np.zeros_like(pb.fixed)                 # no Dirichlet condition at all
    mech = np.zeros_like(pb.fixed).reshape(-1, 3)  # only u_x = 0 on the x = 0 face: a mechanism
    mech[pb.fixed.reshape(-1, 3)[:, 0] != 0, 0] = 1
    return pb, {"no_supports": free, "mechanism": mech.ravel()}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["no_supports", "mechanism"])
def test_singular_problem_reports_and_recovers(precision, case):
    from paper_2201_12931_gb300 import Params, TopoGrid, _lib
    dims = (16, 8, 8)
    pb, masks = _singular_masks(dims)
    g = TopoGrid(dims, Params(levels=3, precision=precision))
    g.set_density(t(synth.uniform_field(dims, 3, 0.1, 1.0)))
    g.set_bc_loads(t(masks[case]), t(pb.f))
    u = torch.full((3 * g.nn,), float("nan"), dtype=torch.float64, device=cuda_device())
    _, res = g.solve(1e-8, 200, out=u, allow_breakdown=True)
    assert res.status in (_lib.TOPO_BREAKDOWN, _lib.TOPO_MAXITER), res
    assert np.isfinite(n(u)).all()
    assert np.isfinite(res.relres) and res.relres > 1e-8
    assert g.lib.topo_last_error(g._h).decode() != ""
    # the same handle, well posed again
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    _, ok = g.solve(1e-8, 2000, out=u)
    assert ok.status == 0 and ok.relres <= 1e-8
    g.close()
