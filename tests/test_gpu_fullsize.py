"""Parity at the benchmark grid sizes, in the launch configuration bench.py times.

* 768x384x384 cantilever (113M elements, the bench workload's grid and 7
  levels): operator rows at sampled nodes (random, corners, clamped face,
  loaded edge, CTA tile seams) on levels 0, 1 and 3, FP64, FP32 and
  double-FP32 kernels,
  against the oracle evaluating the same rows from local data
  (oracle.assemble.operator_rows).  Inputs are drawn from the counter-based
  generator, so the oracle reads the density and vector entries it needs
  directly (raw U[1e-3, 1] density, seed 3; no CUDA output enters the
  oracle).  Mixed-precision solve: compliance within 1e-6 of the FP64 GPU
  solve to 1e-10 (the bench's accuracy claim) and the energy identity.
* 128x64x64 cantilever (the mixed-precision workload): mixed and FP64 GPU
  solves against the oracle's own solve (assembled CSR, Galerkin-MG PCG to
  1e-12): displacement and compliance <= 1e-6, sensitivity <= 1e-5.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import assemble, element, filter as oflt, state as ostate
from gpu_common import cuda_device, n, t

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DIMS = (768, 384, 384)
LEVELS = 7
RHO_SEED, U_SEED = 3, 44


def _rho_at(idx):
    return 1e-3 + (1.0 - 1e-3) * synth.uniform01_at(RHO_SEED, idx)


@pytest.fixture(scope="module")
def big_grid():
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_MIXED
    dev = cuda_device()
    g = TopoGrid(DIMS, Params(levels=LEVELS, precision=TOPO_MIXED))
    ne = DIMS[0] * DIMS[1] * DIMS[2]
    g.set_density(torch.tensor(_rho_at(np.arange(ne)), device=dev))
    pb = synth.cantilever(DIMS)
    g.set_bc_loads(torch.tensor(pb.fixed, device=dev), torch.tensor(pb.f, device=dev))
    del pb
    yield g
    g.close()
    torch.cuda.empty_cache()


def _sample_nodes(dims, count, seed):
    nx, ny, nz = dims
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    nn = NX * NY * NZ
    pts = [(i, j, k) for i in (0, nx) for j in (0, ny) for k in (0, nz)]            # corners
    pts += [(0, ny // 2, nz // 3), (1, 5, 7), (nx, ny // 2, 0), (nx, 3, 0)]         # clamp face, load edge
    pts += [(i, j, nz // 2) for i in (29, 30, 31, 32, 61, 62) for j in (5, 6, 7, 13, 14)]  # CTA seams
    ids = [i + NX * (j + NY * k) for i, j, k in pts if i <= nx and j <= ny and k <= nz]
    ids += list(synth.sample_without_replacement(seed, nn, count))
    return np.asarray(ids, dtype=np.int64)


def _coarse_E(level, dims_l, penal=3.0, E0=1.0, Emin=1e-9):
    """E of level-l elements: SIMP of the mean of the 8^l fine descendants."""
    f = 2 ** level
    nxl, nyl, _ = dims_l
    nx, ny, _ = DIMS

    def E_of(elems):
        out = np.empty(len(elems))
        for q, e in enumerate(elems):
            I, J, K = e % nxl, (e // nxl) % nyl, e // (nxl * nyl)
            a = np.arange(f)
            ii, jj, kk = np.meshgrid(I * f + a, J * f + a, K * f + a, indexing="ij")
            fine = (ii + nx * (jj + ny * kk)).ravel()
            r = _rho_at(fine).mean()
            out[q] = f * (Emin + r ** penal * (E0 - Emin))
        return out
    return E_of


@pytest.mark.parametrize("level", [0, 1, 3])
def test_operator_rows_at_sampled_nodes(big_grid, level):
    g = big_grid
    dims_l = g.level_dims(level)
    nn_l = synth.n_nodes(dims_l)
    seed = U_SEED + level
    u = torch.tensor(synth.uniform01(seed, 3 * nn_l) - 0.5, device=cuda_device())
    y64 = g.apply_operator(u, level=level, precision=0)
    y32 = g.apply_operator(u, level=level, precision=1)
    ydf = g.apply_operator(u, level=level, precision=3)
    nodes = _sample_nodes(dims_l, 300, 45 + level)
    idx = torch.tensor((3 * nodes[:, None] + np.arange(3)).ravel(), device=cuda_device())
    g64 = n(y64[idx]).reshape(-1, 3)
    g32 = n(y32[idx]).reshape(-1, 3)
    gdf = n(ydf[idx]).reshape(-1, 3)
    del u, y64, y32, ydf
    K0 = element.element_stiffness(0.3)
    ref = assemble.operator_rows(dims_l, nodes, _coarse_E(level, dims_l),
                                 lambda d: synth.uniform01_at(seed, d) - 0.5, K0,
                                 lambda d: synth.cantilever_fixed_at(dims_l, d))
    scale = np.abs(ref).max()
    assert np.abs(g64 - ref).max() <= 1e-12 * scale
    assert np.abs(g32 - ref).max() <= 1e-5 * scale
    assert np.abs(gdf - ref).max() <= 1e-12 * scale


def test_mixed_solve_compliance_against_fp64(big_grid):
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_FP64
    g = big_grid
    g.reset_solution()
    _, r = g.solve(1e-6, 5000)
    assert r.status == 0 and r.relres <= 1e-6
    C, _ = g.compliance_and_sensitivity()
    g64 = TopoGrid(DIMS, Params(levels=LEVELS, precision=TOPO_FP64))
    ne = DIMS[0] * DIMS[1] * DIMS[2]
    g64.set_density(torch.tensor(_rho_at(np.arange(ne)), device=cuda_device()))
    pb = synth.cantilever(DIMS)
    f = torch.tensor(pb.f, device=cuda_device())
    g64.set_bc_loads(torch.tensor(pb.fixed, device=cuda_device()), f)
    u = torch.empty(3 * g64.nn, dtype=torch.float64, device=cuda_device())
    _, r64 = g64.solve(1e-10, 5000, out=u)
    assert r64.status == 0
    C64, _ = g64.compliance_and_sensitivity()
    fu = float(torch.dot(f, u))
    g64.close()
    assert abs(C - C64) <= 1e-6 * abs(C64)
    assert abs(C64 - fu) <= 1e-9 * abs(C64)       # energy identity of the FP64 solve


@pytest.mark.parametrize("precision", [0, 1])
def test_cantilever_128x64x64_against_oracle(precision):
    from paper_2201_12931_gb300 import Params, TopoGrid
    name = "cantilever_128x64x64_mixed"
    w = synth.WORKLOADS[name]
    dims = w["dims"]
    pb = synth.make_problem(name)
    rho = oflt.density_filter(synth.raw_density(name), dims, w["density"]["rmin"])
    u_o = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-12, method="mgpcg")
    C_o, _, dc_o = ostate.compliance_and_sensitivity(dims, rho, u_o, pb.f)
    g = TopoGrid(dims, Params(levels=w["levels"], precision=precision))
    g.set_density(t(rho))
    g.set_bc_loads(t(pb.fixed), t(pb.f))
    u = torch.empty(3 * g.nn, dtype=torch.float64, device=cuda_device())
    _, res = g.solve(1e-8, 5000, out=u)
    dc = torch.empty(g.ne, dtype=torch.float64, device=cuda_device())
    C, _ = g.compliance_and_sensitivity(dc)
    assert res.status == 0
    uu = n(u)
    assert np.linalg.norm(uu - u_o) <= 1e-6 * np.linalg.norm(u_o)
    assert abs(C - C_o) <= 1e-6 * abs(C_o)
    assert np.abs(n(dc) - dc_o).max() <= 1e-5 * np.abs(dc_o).max()
