"""Pin of the oracle's local operator rows (used at sampled nodes of grids too
large to assemble) against the assembled Dirichlet operator."""
import numpy as np

import synth
from oracle import assemble, element


def test_local_rows_equal_assembled_rows():
    dims = (5, 4, 3)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 3, 1e-3, 1.0)
    E = assemble.simp_modulus(rho)
    K0 = element.element_stiffness(0.3)
    K = assemble.apply_dirichlet(assemble.assemble(dims, E, K0), pb.fixed)
    u = synth.uniform01(4, pb.f.size) - 0.5
    y = K @ u
    nodes = np.arange(synth.n_nodes(dims))
    rows = assemble.operator_rows(dims, nodes, lambda e: E[e], lambda d: u[d], K0, lambda d: pb.fixed[d])
    assert np.abs(rows.ravel() - y).max() < 1e-14 * np.abs(y).max()


def test_local_rows_without_dirichlet():
    dims = (3, 3, 2)
    E = synth.uniform_field(dims, 9, 0.1, 1.0)
    K0 = element.element_stiffness(0.3)
    K = assemble.assemble(dims, E, K0)
    u = synth.uniform01(5, 3 * synth.n_nodes(dims))
    rows = assemble.operator_rows(dims, [0, 7, 20, 47], lambda e: E[e], lambda d: u[d], K0)
    ref = (K @ u).reshape(-1, 3)[[0, 7, 20, 47]]
    assert np.abs(rows - ref).max() < 1e-14 * np.abs(ref).max()
