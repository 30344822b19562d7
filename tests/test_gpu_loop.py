"""End-to-end GPU checks: the topology-optimisation loop (Algorithm 4 with a
density filter) against the oracle's loop, and the autograd Function rho -> C
against central finite differences and the oracle's full gradient."""
import numpy as np
import pytest
import torch

import synth
from oracle import filter as oflt, state as ostate
from gpu_common import cuda_device, n, t

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_oc_loop_cantilever_48x24x24_20_iterations():
    from paper_2201_12931_gb300 import Params, TopoGrid
    name = "cantilever_48x24x24_fp64_oc20"
    w = synth.WORKLOADS[name]
    dims, oc = w["dims"], w["oc"]
    pb = synth.make_problem(name)
    ne = dims[0] * dims[1] * dims[2]
    x0 = synth.raw_density(name)
    g = TopoGrid(dims, Params(levels=w["levels"]))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    xg = t(x0)
    dc = torch.empty(ne, dtype=torch.float64, device=cuda_device())
    C_gpu, ch_gpu, its = [], [], []
    for _ in range(oc["iters"]):
        g.set_density(g.filter(oc["rmin"], xg))
        _, res = g.solve(1e-10, 3000)
        assert res.status == 0, res
        its.append(res.iters)
        C, _ = g.compliance_and_sensitivity(dc)
        ch_gpu.append(g.oc_update(oc["rmin"], oc["move"], oc["volfrac"], xg, dc))
        C_gpu.append(C)
    xo, u_prev, C_o, ch_o = x0.copy(), None, [], []
    for _ in range(oc["iters"]):
        out = ostate.oc_iteration(dims, xo, pb.fixed, pb.f, oc["rmin"], oc["volfrac"], oc["move"], tol=1e-11,
                                  x0=u_prev)
        C_o.append(out["C"])
        ch_o.append(out["change"])
        xo, u_prev = out["x_new"], out["u"]
    rel = np.abs(np.array(C_gpu) - np.array(C_o)) / np.abs(np.array(C_o))
    print("per-iteration |dC|/C:", " ".join(f"{v:.1e}" for v in rel), "PCG iterations:", its)
    assert np.all(rel[:10] <= 1e-6)
    assert np.all(rel <= 1e-4)
    assert np.abs(n(xg) - xo).max() <= 1e-3
    assert C_gpu[-1] < C_gpu[0]


def test_sensitivity_filter_loop_cantilever_48x24x24():
    """The paper's loop (Algorithm 4 with Eq. sensitivity filter, the design
    as physical density) for 12 iterations against the oracle's loop."""
    from paper_2201_12931_gb300 import Params, TopoGrid
    name = "cantilever_48x24x24_fp64_oc20"
    w = synth.WORKLOADS[name]
    dims, oc = w["dims"], w["oc"]
    iters = 12
    pb = synth.make_problem(name)
    ne = dims[0] * dims[1] * dims[2]
    x0 = synth.raw_density(name)
    g = TopoGrid(dims, Params(levels=w["levels"]))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    xg = t(x0)
    dc = torch.empty(ne, dtype=torch.float64, device=cuda_device())
    C_gpu = []
    for _ in range(iters):
        g.set_density(xg)
        _, res = g.solve(1e-10, 3000)
        assert res.status == 0, res
        C, _ = g.compliance_and_sensitivity(dc)
        dcf = g.sensitivity_filter(oc["rmin"], xg, dc)
        g.oc_update_unfiltered(oc["move"], oc["volfrac"], xg, dcf)
        C_gpu.append(C)
    xo, u_prev, C_o = x0.copy(), None, []
    for _ in range(iters):
        out = ostate.oc_iteration_sensitivity_filter(dims, xo, pb.fixed, pb.f, oc["rmin"], oc["volfrac"],
                                                     oc["move"], tol=1e-11, x0=u_prev)
        C_o.append(out["C"])
        xo, u_prev = out["x_new"], out["u"]
    rel = np.abs(np.array(C_gpu) - np.array(C_o)) / np.abs(np.array(C_o))
    print("per-iteration |dC|/C:", " ".join(f"{v:.1e}" for v in rel))
    assert np.all(rel[:8] <= 1e-6)
    assert np.all(rel <= 1e-4)
    assert C_gpu[-1] < C_gpu[0]


def test_autograd_mbb_96x48x48_fd_and_oracle():
    from paper_2201_12931_gb300 import Params, TopoGrid
    from paper_2201_12931_gb300.autograd import compliance
    name = "mbb_96x48x48_grad"
    w = synth.WORKLOADS[name]
    dims, fd, r = w["dims"], w["fd"], w["density"]["rmin"]
    pb = synth.make_problem(name)
    x = synth.raw_density(name)
    g = TopoGrid(dims, Params(levels=w["levels"]))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    xt = t(x).requires_grad_(True)
    C = compliance(xt, g, r, rel_tol=1e-11)
    C.backward()
    grad = n(xt.grad)
    idx = synth.sample_without_replacement(fd["seed"], x.size, fd["count"])
    h = fd["h"]
    fds = []
    with torch.no_grad():
        for e in idx:
            xp = t(x)
            xp[e] += h
            cp = float(compliance(xp, g, r, rel_tol=1e-11))
            xp[e] -= 2 * h
            cm = float(compliance(xp, g, r, rel_tol=1e-11))
            fds.append((cp - cm) / (2 * h))
    fds = np.array(fds)
    gmax = np.abs(grad).max()
    # FD truncation O(h^2) plus the rounding of C itself (~1e-14 C) divided by 2h
    bound = 1e-5 * gmax + 4e-14 * abs(float(C)) / (2 * h)
    err = np.abs(fds - grad[idx])
    print("max |fd - grad| / max|grad| =", err.max() / gmax)
    assert np.all(err <= bound)
    # oracle's full gradient dC/dx = H^T dc(H x)
    rho = oflt.density_filter(x, dims, r)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-12)
    C_o, _, dc_o = ostate.compliance_and_sensitivity(dims, rho, u_o, pb.f)
    g_o = oflt.density_filter_T(dc_o, dims, r)
    assert abs(float(C) - C_o) <= 1e-9 * abs(C_o)
    assert np.abs(grad - g_o).max() <= 1e-5 * np.abs(g_o).max()
