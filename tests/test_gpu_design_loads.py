"""Non-design regions and the design-dependent self-weight load (Sec. 5,
Examples 2 and 4) on the GPU, against the oracle: the load vector, the
compliance and its sensitivity with the load term, the OC step with passive
elements, and a short loop of the paper's scheme (sensitivity filter) on a
bridge stand-in with both."""
import numpy as np
import pytest
import torch

import synth
from oracle import element, filter as oflt, oc as ooc, sensitivity as osens, state as ostate
from gpu_common import cuda_device, n, rel_max, t

pytestmark = pytest.mark.gpu

DIMS = (32, 8, 16)
W = 0.05


def _bridge():
    return synth.arch_bridge(DIMS, deck_layers=2, slot_halfwidth=1.5, q=1.0)


def test_gravity_load_compliance_and_sensitivity():
    from paper_2201_12931_gb300 import Params, TopoGrid
    pb = _bridge()
    pas = pb.info["passive"]
    rho = synth.uniform_field(DIMS, 71, 0.1, 1.0)
    rho[pas == 1], rho[pas == 2] = 1.0, 1e-3
    g = TopoGrid(DIMS, Params(levels=3))
    f_gpu = g.gravity_load(W, t(rho), t(pb.f))
    f_o = osens.gravity_load(DIMS, rho, W, pb.f)
    assert rel_max(n(f_gpu), f_o) < 1e-14
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), f_gpu)
    _, res = g.solve(1e-10, 3000)     # point supports: the FP64 floor is ~1e-11
    assert res.status == 0
    dc = torch.empty(g.ne, dtype=torch.float64, device=cuda_device())
    C, _ = g.compliance_and_sensitivity(dc)
    g.gravity_sensitivity(W, dc)
    u_o = ostate.solve_state(DIMS, rho, pb.fixed, f_o, tol=1e-13)
    C_o, _, dc_o = ostate.compliance_and_sensitivity(DIMS, rho, u_o, np.where(pb.fixed.astype(bool), 0.0, f_o))
    dc_o = dc_o + osens.gravity_sensitivity_term(DIMS, u_o, W)
    assert abs(C - C_o) <= 1e-8 * abs(C_o)
    assert rel_max(n(dc), dc_o) < 1e-6


def test_oc_update_with_passive_elements():
    from paper_2201_12931_gb300 import Params, TopoGrid
    pas = _bridge().info["passive"]
    g = TopoGrid(DIMS, Params(levels=1))
    x = synth.uniform_field(DIMS, 72, 0.1, 0.5)
    x[pas == 1], x[pas == 2] = 1.0, 0.0
    dc = synth.uniform_field(DIMS, 73, -5.0, 0.5)      # some positive entries (load term)
    xg = t(x)
    ch = g.oc_update_unfiltered(0.2, 0.2, xg, t(dc), passive=t(pas))
    xo, cho, _, _ = ooc.oc_update_unfiltered(x, dc, 0.2, 0.2, passive=pas)
    assert np.abs(n(xg) - xo).max() < 1e-7
    assert abs(ch - cho) < 1e-7
    assert np.all(n(xg)[pas == 1] == 1.0) and np.all(n(xg)[pas == 2] == 0.0)


def test_bridge_loop_with_passive_regions_and_self_weight():
    """Six iterations of Algorithm 4 with the sensitivity filter, passive
    deck and slot, pressure on the deck plus self-weight, against the
    oracle's loop."""
    from paper_2201_12931_gb300 import Params, TopoGrid
    pb = _bridge()
    pas = pb.info["passive"]
    vf, r, move, iters = 0.2, 1.5, 0.2, 6
    x0 = np.full(pas.size, vf)
    x0[pas == 1], x0[pas == 2] = 1.0, 0.0
    g = TopoGrid(DIMS, Params(levels=3))
    fixed_d, fext_d, pas_d = t(pb.fixed), t(pb.f), t(pas)
    xg = t(x0)
    dc = torch.empty(g.ne, dtype=torch.float64, device=cuda_device())
    C_gpu = []
    for _ in range(iters):
        g.set_density(xg)
        g.set_bc_loads(fixed_d, g.gravity_load(W, xg, fext_d))
        _, res = g.solve(1e-10, 3000)
        assert res.status == 0, res
        C, _ = g.compliance_and_sensitivity(dc)
        g.gravity_sensitivity(W, dc)
        g.oc_update_unfiltered(move, vf, xg, g.sensitivity_filter(r, xg, dc), passive=pas_d)
        C_gpu.append(C)
    x, C_o, u_prev = x0.copy(), [], None
    for _ in range(iters):
        f = osens.gravity_load(DIMS, x, W, pb.f)
        u = ostate.solve_state(DIMS, x, pb.fixed, f, tol=1e-12, x0=u_prev)
        C, _, dco = ostate.compliance_and_sensitivity(DIMS, x, u, np.where(pb.fixed.astype(bool), 0.0, f))
        dco = dco + osens.gravity_sensitivity_term(DIMS, u, W)
        x = ooc.oc_update_unfiltered(x, oflt.sensitivity_filter(x, dco, DIMS, r), vf, move, passive=pas)[0]
        C_o.append(C)
        u_prev = u
    rel = np.abs(np.array(C_gpu) - np.array(C_o)) / np.abs(np.array(C_o))
    print("per-iteration |dC|/C:", " ".join(f"{v:.1e}" for v in rel))
    assert np.all(rel <= 1e-6)
    assert np.abs(n(xg) - x).max() <= 1e-4
