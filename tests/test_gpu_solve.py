"""GPU state solve, compliance and sensitivity against the oracle.

Bars: relative L2 displacement error and relative compliance error <= 1e-6
at rel_tol 1e-8, and <= 1e-9 at rel_tol 1e-12 (FP64 path); sensitivity max
error <= 1e-7 relative to max |dc| (FP64 path).  Mixed-precision handles
reach the same displacement bars (the FP64 refinement loop reaches the FP64
residual target) and contract the element energy in FP32 after an FP64
translation shift: compliance <= 1e-7, sensitivity <= 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import filter as oflt, state as ostate
from gpu_common import cuda_device, n, t

pytestmark = pytest.mark.gpu


def _gpu_solve(dims, levels, problem, rho, precision, tol, **kw):
    from paper_2201_12931_gb300 import Params, TopoGrid
    import torch
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    g = TopoGrid(dims, Params(levels=levels, precision=precision, **kw))
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
    _, res = g.solve(tol, 2000, out=u)
    dc = torch.empty(g.ne, dtype=torch.float64, device=cuda_device())
    C, _ = g.compliance_and_sensitivity(dc)
    return g, pb, n(u), C, n(dc), res


@pytest.mark.parametrize("dims,levels,problem", [
    ((48, 24, 24), 3, "cantilever"),
    ((32, 16, 16), 4, "mbb"),
    ((12, 4, 4), 1, "cantilever"),
])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_solve_matches_oracle(dims, levels, problem, precision):
    rho = synth.uniform_field(dims, 1, 1e-3, 1.0)
    rho = oflt.density_filter(rho, dims, 1.5)
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    C_o, _, dc_o = ostate.compliance_and_sensitivity(dims, rho, u_o, pb.f)
    for tol, bar in ((1e-8, 1e-6), (1e-12, 1e-9)):
        g, _, u, C, dc, res = _gpu_solve(dims, levels, problem, rho, precision, tol)
        assert res.status == 0, res
        assert res.relres <= tol
        assert np.linalg.norm(u - u_o) <= bar * np.linalg.norm(u_o)
        # FP64 path: the solve's bar; mixed handles contract the element
        # energy in FP32 (bars 1e-7 on C, 1e-5 on dc, stated per result)
        c_bar = bar if precision == 0 else max(bar, 1e-7)
        dc_bar = max(bar, 1e-7) if precision == 0 else 1e-5
        assert abs(C - C_o) <= c_bar * abs(C_o)
        assert np.abs(dc - dc_o).max() <= dc_bar * np.abs(dc_o).max()
        # energy identity C = f^T u on the GPU result
        assert abs(C - pb.f @ u) <= max(10 * tol, 0.0 if precision == 0 else 1e-7) * abs(C)


@pytest.mark.parametrize("dims,levels,problem", [((48, 24, 24), 3, "cantilever"), ((32, 16, 16), 4, "mbb")])
@pytest.mark.parametrize("homogenize", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_coarsening_variants_reach_the_oracle_solution(dims, levels, problem, homogenize, precision):
    """The coarse operators only precondition: with the modulus-averaging
    and the stored Galerkin coarse operators the solve reaches the oracle's
    displacement (1e-6 at rel. residual 1e-8) and compliance."""
    rho = oflt.density_filter(synth.uniform_field(dims, 1, 1e-3, 1.0), dims, 1.5)
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    C_o, _, _ = ostate.compliance_and_sensitivity(dims, rho, u_o, pb.f)
    g, _, u, C, dc, res = _gpu_solve(dims, levels, problem, rho, precision, 1e-8, homogenize=homogenize)
    assert res.status == 0 and res.relres <= 1e-8
    assert np.linalg.norm(u - u_o) <= 1e-6 * np.linalg.norm(u_o)
    assert abs(C - C_o) <= (1e-6 if precision == 0 else 1e-7 + 1e-6) * abs(C_o)


def test_uniform_density_cantilever_48():
    dims = (48, 24, 24)
    rho = np.full(27648, 0.3)
    pb = synth.cantilever(dims)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    g, _, u, C, dc, res = _gpu_solve(dims, 3, "cantilever", rho, 0, 1e-8)
    assert res.status == 0 and res.iters < 60
    assert np.linalg.norm(u - u_o) <= 1e-6 * np.linalg.norm(u_o)


def test_warm_start_reduces_iterations():
    dims = (16, 8, 8)
    rho = synth.uniform_field(dims, 2, 0.1, 1.0)
    from paper_2201_12931_gb300 import Params, TopoGrid
    pb = synth.cantilever(dims)
    g = TopoGrid(dims, Params(levels=3))
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    _, r1 = g.solve(1e-8, 500)
    _, r2 = g.solve(1e-8, 500)
    assert r2.iters == 0 and r2.relres <= 1e-8


def test_zero_load_gives_zero_solution():
    dims = (8, 4, 4)
    from paper_2201_12931_gb300 import Params, TopoGrid
    import torch
    pb = synth.cantilever(dims)
    g = TopoGrid(dims, Params(levels=2))
    g.set_density(t(np.full(128, 0.5)))
    g.set_bc_loads(t(pb.fixed), t(np.zeros_like(pb.f)))
    u = torch.ones(3 * g.nn, dtype=torch.float64, device=cuda_device())
    _, res = g.solve(1e-8, 100, out=u)
    assert res.status == 0 and float(u.abs().max()) == 0.0


def test_bad_density_is_rejected():
    dims = (8, 4, 4)
    from paper_2201_12931_gb300 import Params, TopoError, TopoGrid
    pb = synth.cantilever(dims)
    g = TopoGrid(dims, Params(levels=2))
    rho = np.full(128, 0.5)
    rho[7] = np.nan
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    with pytest.raises(TopoError):
        g.solve(1e-8, 100)


def test_maxiter_reported():
    dims = (16, 8, 8)
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_MAXITER
    pb = synth.cantilever(dims)
    g = TopoGrid(dims, Params(levels=2))
    g.set_density(t(synth.uniform_field(dims, 3, 1e-3, 1.0)))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    _, res = g.solve(1e-14, 2)
    assert res.status == TOPO_MAXITER and res.iters == 2


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_replay_is_bitwise_identical(precision):
    """PCG iterations replayed from the captured CUDA graph launch the same
    kernels in the same order as direct launches: identical results."""
    from paper_2201_12931_gb300 import Params, TopoGrid
    import torch
    dims, levels = (48, 24, 24), 3
    rho = oflt.density_filter(synth.uniform_field(dims, 1, 1e-3, 1.0), dims, 1.5)
    pb = synth.cantilever(dims)
    out = []
    for graphs in (1, 0):
        g = TopoGrid(dims, Params(levels=levels, precision=precision, graphs=graphs))
        g.set_density(t(rho))
        g.set_bc_loads(t(pb.fixed), t(pb.f))
        u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
        _, res = g.solve(1e-10, 2000, out=u)
        assert res.status == 0
        out.append((n(u), res))
    (u1, r1), (u0, r0) = out
    assert r1.graph_replays > 0 and r0.graph_replays == 0
    assert r1.iters == r0.iters
    assert np.array_equal(u1, u0)


def test_direction_ring_wraps_and_flushes():
    """The CG directions live in a ring of 8 buffers and x += alpha p is
    applied once per full ring (inside the captured iteration of slot 7) and
    for the remainder when the run stops.  A single FP64 CG run of more than
    two ring lengths, with graphs and with direct launches, reaches the
    oracle's solution and both runs agree bitwise; a run stopped after 11
    steps (one full ring and 3 more) returns an x whose FP64 residual,
    recomputed from the oracle's assembled K, is the one it reports."""
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_MAXITER
    from oracle import assemble, element
    import torch
    dims, levels = (32, 16, 16), 2     # two levels: slow enough for > 16 iterations
    rho = synth.uniform_field(dims, 7, 1e-3, 1.0)
    pb = synth.cantilever(dims)
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-13)
    K = assemble.apply_dirichlet(assemble.assemble(dims, assemble.simp_modulus(rho, 1.0, 1e-9, 3.0),
                                                   element.element_stiffness(0.3)), pb.fixed)
    out = []
    for graphs in (1, 0):
        g = TopoGrid(dims, Params(levels=levels, precision=0, graphs=graphs))
        g.set_density(t(rho))
        g.set_bc_loads(t(pb.fixed), t(pb.f))
        u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
        _, res = g.solve(1e-11, 2000, out=u)
        assert res.status == 0 and res.iters > 16, res
        out.append(n(u))
        g.reset_solution()
        u2 = torch.empty_like(u)
        _, r2 = g.solve(1e-14, 11, out=u2)
        assert r2.status == TOPO_MAXITER and r2.iters == 11
        rr = np.linalg.norm(pb.f - K @ n(u2)) / np.linalg.norm(pb.f)
        assert abs(rr - r2.relres) <= 1e-6 * rr
        g.close()
    assert np.array_equal(out[0], out[1])
    assert np.linalg.norm(out[0] - u_o) <= 1e-8 * np.linalg.norm(u_o)
