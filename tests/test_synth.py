"""Pins of the shared seeded input generators (no method arithmetic here)."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_outputs():
    with open(os.path.join(GOLDEN, "splitmix64.json")) as fh:
        g = json.load(fh)
    got = [int(v) for v in synth.splitmix64(g["seed"], 3)]
    assert got == [int(h, 16) for h in g["outputs_hex"]]


def test_uniform_range_and_determinism():
    a = synth.uniform_field((8, 4, 4), 1, 1e-3, 1.0)
    b = synth.uniform_field((8, 4, 4), 1, 1e-3, 1.0)
    assert np.array_equal(a, b)
    assert a.min() >= 1e-3 and a.max() < 1.0
    assert abs(synth.uniform01(5, 100000).mean() - 0.5) < 0.01


def test_cantilever_load_resultant_and_clamp():
    pb = synth.cantilever((6, 4, 2))
    assert pb.f.sum() == -4.0
    fx = pb.fixed.reshape(-1, 3)
    assert fx.sum() == 3 * 5 * 3


def test_mbb_constraints():
    pb = synth.mbb_half((6, 4, 2))
    fx = pb.fixed.reshape(-1, 3)
    assert fx[:, 0].sum() == 5 * 3 and fx[:, 2].sum() == 5 and fx[:, 1].sum() == 1
    assert pb.f.sum() == -4.0


def test_sample_without_replacement():
    s = synth.sample_without_replacement(2, 1000, 64)
    assert len(set(s.tolist())) == 64 and s.min() >= 0 and s.max() < 1000


def test_uniform01_at_matches_stream():
    idx = np.array([0, 5, 99, 12345, 7])
    assert np.array_equal(synth.uniform01_at(9, idx), synth.uniform01(9, 20000)[idx])


def test_cantilever_fixed_at_matches_mask():
    dims = (5, 3, 2)
    pb = synth.cantilever(dims)
    dofs = np.arange(pb.fixed.size)
    assert np.array_equal(synth.cantilever_fixed_at(dims, dofs), pb.fixed)


def test_arch_bridge_regions_and_loads():
    dims = (32, 8, 16)
    pb = synth.arch_bridge(dims, deck_layers=2, slot_halfwidth=1.5, q=2.0)
    pas = pb.info["passive"].reshape(16, 8, 32)
    assert np.all(pas[14:] == 1)
    assert np.all(pas[:8, :, 14:18] == 2) and np.all(pas[8:14, :, 14:18] == 0)
    assert np.all(pas[:14, :, :14] == 0) and np.all(pas[:14, :, 18:] == 0)
    assert pb.f[2::3].sum() == pytest.approx(-2.0 * 32 * 8)      # resultant of the pressure
    assert pb.fixed.sum() == 2 * 9 + 9 + 1


@pytest.mark.parametrize("name", sorted(synth.WORKLOADS))
def test_workload_hierarchies_are_valid(name):
    """Every named workload's grid divides by 2^(levels-1) and its coarsest
    grid fits the dense direct solve (at most 12000 DOFs)."""
    w = synth.WORKLOADS[name]
    nx, ny, nz = w["dims"]
    f = 2 ** (w["levels"] - 1)
    assert nx % f == 0 and ny % f == 0 and nz % f == 0
    ndof = 3 * (nx // f + 1) * (ny // f + 1) * (nz // f + 1)
    assert ndof <= 12000, ndof
