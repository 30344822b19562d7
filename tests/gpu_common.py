"""Helpers shared by the GPU parity tests: build both sides from the same
seeded synthetic inputs (synth), never feeding a CUDA result to the oracle."""
from __future__ import annotations

import numpy as np

import synth
from oracle import element, multigrid


def cuda_device():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch.device("cuda", 0)


def make_case(dims, levels, problem="cantilever", seed=3, lo=1e-3, hi=1.0, precision=0, **kw):
    """Returns (grid, problem, rho (numpy), oracle hierarchy)."""
    import torch
    from paper_2201_12931_gb300 import Params, TopoGrid
    dev = cuda_device()
    pb = synth.cantilever(dims) if problem == "cantilever" else synth.mbb_half(dims)
    rho = synth.uniform_field(dims, seed, lo, hi)
    g = TopoGrid(dims, Params(levels=levels, precision=precision, **kw))
    g.set_density(torch.tensor(rho, device=dev))
    g.set_bc_loads(torch.tensor(pb.fixed, device=dev), torch.tensor(pb.f, device=dev))
    K0 = element.element_stiffness(g.params.nu)
    if g.params.homogenize == 2:
        from oracle import assemble
        E = assemble.simp_modulus(rho, g.params.E0, g.params.Emin, g.params.penal)
        K = assemble.apply_dirichlet(assemble.assemble(dims, E, K0), pb.fixed)
        H = multigrid.galerkin_hierarchy(dims, K, pb.fixed, levels)
        return g, pb, rho, H
    rule = "modulus" if g.params.homogenize == 1 else "density"
    H = multigrid.homogenized_hierarchy(dims, rho, pb.fixed, K0, levels, g.params.E0, g.params.Emin,
                                        g.params.penal, rule=rule)
    return g, pb, rho, H


def t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device=cuda_device())


def n(x):
    return x.detach().cpu().numpy()


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
