"""Pins of the oracle's density filter, its transpose, the sensitivity and
the OC update.

* filter: a constant field maps to itself, interior neighbour counts from
  the lattice (golden), agreement with an O(N^2) brute-force loop, and the
  dot-product test <H a, b> = <a, H^T b>;
* sensitivity: central finite differences of c(rho) = f^T u(rho) with dense
  direct solves;
* OC: move limits and box bounds hold, the volume constraint is met to the
  bisection tolerance, and the update keeps x where B = 1.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import assemble, element, filter as flt, oc, sensitivity, solve, state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("r", [1.5, 2.0, 2.5, 3.0])
def test_filter_preserves_constants(r):
    dims = (7, 5, 4)
    out = flt.density_filter(np.full(140, 0.37), dims, r)
    assert np.abs(out - 0.37).max() < 1e-15


def test_neighbour_counts_golden():
    with open(os.path.join(GOLDEN, "filter_neighbours.json")) as fh:
        g = json.load(fh)
    for r, n in g["counts"].items():
        assert len(flt.offsets(float(r))) == n


@pytest.mark.parametrize("r", [1.5, 2.0, 2.5])
def test_filter_matches_bruteforce(r):
    dims = (5, 4, 3)
    x = synth.uniform_field(dims, 21)
    assert np.abs(flt.density_filter(x, dims, r) - flt.density_filter_bruteforce(x, dims, r)).max() < 1e-14


@pytest.mark.parametrize("r", [1.5, 3.0])
def test_filter_transpose_dot_product(r):
    dims = (6, 5, 4)
    a = synth.uniform_field(dims, 1)
    b = synth.uniform_field(dims, 2, -1.0, 1.0)
    lhs = flt.density_filter(a, dims, r) @ b
    rhs = a @ flt.density_filter_T(b, dims, r)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def _compliance(dims, rho, pb):
    u = state.solve_state(dims, rho, pb.fixed, pb.f, method="dense")
    return pb.f @ u, u


def test_sensitivity_central_differences():
    dims = (4, 2, 2)
    pb = synth.cantilever(dims)
    rho = synth.uniform_field(dims, 13, 0.2, 1.0)
    C, u = _compliance(dims, rho, pb)
    _, C2, dc = state.compliance_and_sensitivity(dims, rho, u, pb.f)
    assert C2 == pytest.approx(C, rel=1e-12)
    h = 1e-5
    for e in range(rho.size):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (_compliance(dims, rp, pb)[0] - _compliance(dims, rm, pb)[0]) / (2 * h)
        assert fd == pytest.approx(dc[e], rel=1e-6, abs=1e-9 * np.abs(dc).max())


def test_sensitivity_mbb_with_filter_chain_rule():
    """dc/dx = H^T dc/drho~ against finite differences through the filter."""
    dims = (4, 2, 2)
    pb = synth.mbb_half(dims)
    x = synth.uniform_field(dims, 17, 0.3, 1.0)
    r = 1.5

    def C_of(xv):
        rho = flt.density_filter(xv, dims, r)
        return _compliance(dims, rho, pb)[0]

    rho = flt.density_filter(x, dims, r)
    _, u = _compliance(dims, rho, pb)
    _, _, dc = state.compliance_and_sensitivity(dims, rho, u, pb.f)
    g = flt.density_filter_T(dc, dims, r)
    h = 1e-5
    for e in (0, 5, 11, 15):
        xp, xm = x.copy(), x.copy()
        xp[e] += h
        xm[e] -= h
        fd = (C_of(xp) - C_of(xm)) / (2 * h)
        assert fd == pytest.approx(g[e], rel=1e-6)


def test_oc_bounds_and_volume():
    dims = (8, 4, 4)
    r, vf, move = 1.5, 0.3, 0.2
    x = np.full(128, 0.3)
    dc = -synth.uniform_field(dims, 3, 0.1, 10.0)
    xn, ch, lam, steps = oc.oc_update(x, dc, dims, r, vf, move)
    assert np.all(xn >= 0.0) and np.all(xn <= 1.0)
    assert np.all(xn >= x - move - 1e-15) and np.all(xn <= x + move + 1e-15)
    assert abs(flt.density_filter(xn, dims, r).mean() - vf) < 1e-6
    assert ch == pytest.approx(np.abs(xn - x).max())
    assert 40 < steps < 80


def test_oc_fixed_point_when_kkt_holds():
    """If -dc~ = lambda dv~ for the lambda the bisection finds, x is unchanged."""
    dims = (6, 4, 4)
    r = 2.0
    x = np.full(96, 0.4)
    dvt = flt.density_filter_T(np.ones(96), dims, r)
    # dc chosen so that H^T dc = -2.5 * H^T 1, i.e. dc = -2.5 * ones
    dc = -2.5 * np.ones(96)
    xn, ch, lam, _ = oc.oc_update(x, dc, dims, r, volfrac=0.4, move=0.2)
    assert lam == pytest.approx(2.5, rel=1e-6)
    assert ch < 1e-6


@pytest.mark.parametrize("r", [1.5, 2.5])
def test_sensitivity_filter_matches_bruteforce(r):
    """Eq. sensitivity filter against the O(N^2) pair loop applied to rho*dc,
    divided by max(gamma, rho); densities below gamma exercise the clamp."""
    dims = (5, 4, 3)
    rho = synth.uniform_field(dims, 31, 0.0, 1.0)
    rho[::7] = 1e-4                                   # below gamma = 1e-3
    dc = -synth.uniform_field(dims, 32, 0.1, 5.0)
    got = flt.sensitivity_filter(rho, dc, dims, r, gamma=1e-3)
    ref = flt.density_filter_bruteforce(rho * dc, dims, r) / np.maximum(1e-3, rho)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_sensitivity_filter_constant_fields():
    """Uniform density and sensitivity are reproduced exactly (up to rounding)."""
    dims = (6, 5, 4)
    rho = np.full(120, 0.37)
    dc = np.full(120, -2.5)
    got = flt.sensitivity_filter(rho, dc, dims, 2.0)
    assert np.allclose(got, -2.5, rtol=1e-14, atol=0)


def test_oc_unfiltered_bounds_and_volume():
    dims = (8, 4, 4)
    vf, move = 0.3, 0.2
    x = np.full(128, 0.3)
    dc = -synth.uniform_field(dims, 3, 0.1, 10.0)
    xn, ch, lam, steps = oc.oc_update_unfiltered(x, dc, vf, move)
    assert np.all(xn >= 0.0) and np.all(xn <= 1.0)
    assert np.all(xn >= x - move - 1e-15) and np.all(xn <= x + move + 1e-15)
    assert abs(xn.mean() - vf) < 1e-6
    assert ch == pytest.approx(np.abs(xn - x).max())


def test_oc_unfiltered_equals_filtered_oc_with_identity_filter():
    """For r <= 1 the density filter is the identity (only the element itself
    has positive weight), so the filtered OC step reduces to the unfiltered
    one."""
    dims = (6, 4, 4)
    x = synth.uniform_field(dims, 5, 0.1, 0.9)
    dc = -synth.uniform_field(dims, 6, 0.1, 10.0)
    a = oc.oc_update(x, dc, dims, 0.9, 0.45, 0.2)
    b = oc.oc_update_unfiltered(x, dc, 0.45, 0.2)
    assert np.abs(a[0] - b[0]).max() < 1e-12
    assert a[2] == pytest.approx(b[2], rel=1e-12)


def test_oc_unfiltered_passive_elements():
    dims = (8, 4, 4)
    x = np.full(128, 0.3)
    passive = np.zeros(128, dtype=np.uint8)
    passive[:16] = 1                 # solid slab
    passive[60:70] = 2               # void slot
    x[passive == 1], x[passive == 2] = 1.0, 0.0
    dc = -synth.uniform_field(dims, 3, 0.1, 10.0)
    xn, ch, lam, steps = oc.oc_update_unfiltered(x, dc, 0.3, 0.2, passive=passive)
    assert np.all(xn[passive == 1] == 1.0) and np.all(xn[passive == 2] == 0.0)
    assert abs(xn[passive == 0].mean() - 0.3) < 1e-6
    same = oc.oc_update_unfiltered(x, dc, 0.3, 0.2, passive=np.zeros(128, dtype=np.uint8))
    plain = oc.oc_update_unfiltered(x, dc, 0.3, 0.2)
    assert np.array_equal(same[0], plain[0])
