"""GPU parity of every hot-path step against the CPU oracle, through the C-ABI.

Sizes span several CUDA blocks and ragged tails; inputs are seeded synthetic
fields.  Tolerances: FP64 kernels 1e-12 (operators, transfers, filter) and
1e-10 (V-cycle, which stacks ~20 kernel applications) relative to the max
norm of the oracle result; FP32 kernels 1e-5 relative.
"""
import numpy as np
import pytest

import synth
from oracle import element, filter as oflt, multigrid, oc as ooc
from gpu_common import make_case, n, rel_max, t

pytestmark = pytest.mark.gpu

CASES = [((6, 4, 4), 2), ((10, 6, 4), 2), ((13, 7, 5), 1), ((48, 24, 24), 3), ((40, 24, 16), 4)]


@pytest.mark.parametrize("dims,levels", CASES)
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_operator_all_levels(dims, levels, precision, tol):
    g, pb, rho, H = make_case(dims, levels)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 100 + l, -1.0, 1.0)
        y = n(g.apply_operator(t(u), level=l, precision=precision))
        assert rel_max(y, H[l].K @ u) < tol, (l, rel_max(y, H[l].K @ u))


@pytest.mark.parametrize("dims,levels", CASES[:4])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_jacobi_and_residual(dims, levels, precision, tol):
    g, pb, rho, H = make_case(dims, levels, seed=8)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 7, -1.0, 1.0)
        f = synth.uniform_field((nl, 1, 1), 9, -1.0, 1.0)
        f[H[l].fixed.astype(bool)] = 0.0
        uj = n(g.jacobi_sweep(t(u), t(f), level=l, precision=precision))
        ref = multigrid.jacobi(H[l], u, f, g.params.omega)
        assert rel_max(uj, ref) < tol
        r = n(g.residual(t(u), t(f), level=l, precision=precision))
        assert rel_max(r, f - H[l].K @ u) < tol


@pytest.mark.parametrize("dims,levels", [((6, 4, 4), 2), ((48, 24, 24), 3), ((16, 8, 8), 4)])
@pytest.mark.parametrize("problem", ["cantilever", "mbb"])
def test_transfers_and_homogenized_density(dims, levels, problem):
    g, pb, rho, H = make_case(dims, levels, problem=problem)
    for l in range(levels):
        assert rel_max(n(g.level_density(l)), H[l].rho) < 1e-14
    for l in range(levels - 1):
        nf, nc = H[l].K.shape[0], H[l + 1].K.shape[0]
        rf = synth.uniform_field((nf, 1, 1), 31, -1, 1)
        rc = n(g.restrict(t(rf), level=l))
        assert rel_max(rc, H[l].P.T @ rf) < 1e-14
        ec = synth.uniform_field((nc, 1, 1), 32, -1, 1)
        uf = synth.uniform_field((nf, 1, 1), 33, -1, 1)
        out = n(g.prolong_add(t(ec), t(uf), level=l))
        assert rel_max(out, uf + H[l].P @ ec) < 1e-14


@pytest.mark.parametrize("dims,levels", [((8, 4, 4), 2), ((48, 24, 24), 3), ((32, 16, 16), 4)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_vcycle(dims, levels, precision, tol):
    g, pb, rho, H = make_case(dims, levels, seed=4)
    r = synth.uniform_field((H[0].K.shape[0], 1, 1), 12, -1, 1)
    r[pb.fixed.astype(bool)] = 0.0
    z = n(g.vcycle(t(r), precision=precision))
    ref = multigrid.vcycle(H, r, g.params.omega, g.params.pre, g.params.post)
    assert rel_max(z, ref) < tol, rel_max(z, ref)


@pytest.mark.parametrize("dims,levels", [((8, 4, 4), 2), ((48, 24, 24), 3), ((32, 16, 16), 4), ((6, 4, 4), 1)])
def test_vcycle_bf16_iterates(dims, levels):
    """V-cycle with BF16 iterates (FP32 arithmetic) against the oracle's FP64
    V-cycle.  Each stored iterate is rounded to 8 significant bits (relative
    2^-9); along one V-cycle an entry passes through at most pre + post + 1
    roundings per level, so the relative 2-norm error stays below ~20 * 2^-9
    = 0.04.  With one level the V-cycle is the FP32 direct solve (1e-4)."""
    g, pb, rho, H = make_case(dims, levels, seed=4)
    r = synth.uniform_field((H[0].K.shape[0], 1, 1), 12, -1, 1)
    r[pb.fixed.astype(bool)] = 0.0
    z = n(g.vcycle(t(r), precision=2))
    ref = multigrid.vcycle(H, r, g.params.omega, g.params.pre, g.params.post)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err < (1e-4 if levels == 1 else 4e-2), err
    if levels > 1:
        z32 = n(g.vcycle(t(r), precision=1))
        assert np.linalg.norm(z32 - ref) / np.linalg.norm(ref) < err   # the rounding is visible
    assert float(z @ r) > 0.0                                           # still a descent direction


@pytest.mark.parametrize("dims,levels", [((48, 24, 24), 3), ((40, 24, 16), 4)])
def test_modulus_averaging_variant(dims, levels):
    """Coarse moduli = mean of the children's moduli (homogenize = 1): the
    operators of every level and the V-cycle against the oracle's hierarchy
    built with the same rule."""
    g, pb, rho, H = make_case(dims, levels, seed=6, lo=0.0, hi=1.0, homogenize=1)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 200 + l, -1.0, 1.0)
        assert rel_max(n(g.apply_operator(t(u), level=l, precision=0)), H[l].K @ u) < 1e-12
        assert rel_max(n(g.apply_operator(t(u), level=l, precision=1)), H[l].K @ u) < 1e-5
    r = synth.uniform_field((H[0].K.shape[0], 1, 1), 13, -1, 1)
    r[pb.fixed.astype(bool)] = 0.0
    ref = multigrid.vcycle(H, r, g.params.omega, g.params.pre, g.params.post)
    assert rel_max(n(g.vcycle(t(r), precision=0)), ref) < 1e-10


@pytest.mark.parametrize("dims,levels,problem", [((8, 4, 4), 2, "cantilever"), ((48, 24, 24), 3, "cantilever"),
                                                 ((40, 24, 16), 4, "cantilever"), ((32, 16, 16), 3, "mbb")])
def test_galerkin_levels(dims, levels, problem):
    """Stored Galerkin coarse element matrices (homogenize = 2): every
    level's operator, Jacobi sweep and residual, and the V-cycle, against the
    oracle's assembled Galerkin hierarchy P~^T K P~ (FP64 1e-12 / 1e-10,
    FP32 1e-5 / 1e-4)."""
    g, pb, rho, H = make_case(dims, levels, problem=problem, seed=6, lo=1e-3, hi=1.0, homogenize=2)
    for l in range(levels):
        nl = H[l].K.shape[0]
        u = synth.uniform_field((nl, 1, 1), 300 + l, -1.0, 1.0)
        f = synth.uniform_field((nl, 1, 1), 310 + l, -1.0, 1.0)
        f[H[l].fixed.astype(bool)] = 0.0
        ref = H[l].K @ u
        assert rel_max(n(g.apply_operator(t(u), level=l, precision=0)), ref) < 1e-12, l
        assert rel_max(n(g.apply_operator(t(u), level=l, precision=1)), ref) < 1e-5, l
        assert rel_max(n(g.jacobi_sweep(t(u), t(f), level=l, precision=0)),
                       multigrid.jacobi(H[l], u, f, g.params.omega)) < 1e-12, l
        assert rel_max(n(g.residual(t(u), t(f), level=l, precision=0)), f - ref) < 1e-12, l
    r = synth.uniform_field((H[0].K.shape[0], 1, 1), 14, -1, 1)
    r[pb.fixed.astype(bool)] = 0.0
    ref = multigrid.vcycle(H, r, g.params.omega, g.params.pre, g.params.post)
    assert rel_max(n(g.vcycle(t(r), precision=0)), ref) < 1e-10
    assert rel_max(n(g.vcycle(t(r), precision=1)), ref) < 1e-4


@pytest.mark.parametrize("r", [1.5, 2.0, 2.5, 3.0])
@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 9)])
def test_filter_and_transpose(r, dims):
    from paper_2201_12931_gb300 import Params, TopoGrid
    g = TopoGrid(dims, Params(levels=1))
    x = synth.uniform_field(dims, 41)
    y = n(g.filter(r, t(x)))
    assert rel_max(y, oflt.density_filter(x, dims, r)) < 1e-14
    yt = n(g.filter(r, t(x), transpose=True))
    assert rel_max(yt, oflt.density_filter_T(x, dims, r)) < 1e-14


@pytest.mark.parametrize("dims,r", [((12, 6, 6), 1.5), ((20, 10, 8), 2.5)])
def test_oc_update_given_dc(dims, r):
    """OC step from the same x and dc (both synthetic): bisection is decided in
    FP64 on both sides; x_new agrees to the bisection tolerance."""
    from paper_2201_12931_gb300 import Params, TopoGrid
    g = TopoGrid(dims, Params(levels=1))
    x = synth.uniform_field(dims, 51, 0.1, 0.6)
    dc = -synth.uniform_field(dims, 52, 0.01, 5.0)
    xg = t(x)
    ch = g.oc_update(r, 0.2, 0.35, xg, t(dc))
    xo, cho, lam, steps = ooc.oc_update(x, dc, dims, r, 0.35, 0.2)
    assert np.abs(n(xg) - xo).max() < 1e-7
    assert abs(ch - cho) < 1e-7


@pytest.mark.parametrize("r", [1.5, 2.5, 3.0])
@pytest.mark.parametrize("dims", [(7, 5, 3), (33, 17, 9)])
def test_sensitivity_filter(r, dims):
    """Eq. sensitivity filter against the oracle (FP64, 1e-13), densities
    below gamma included."""
    from paper_2201_12931_gb300 import Params, TopoGrid
    g = TopoGrid(dims, Params(levels=1))
    rho = synth.uniform_field(dims, 61, 0.0, 1.0)
    rho[::5] = 2e-4
    dc = -synth.uniform_field(dims, 62, 0.01, 5.0)
    got = n(g.sensitivity_filter(r, t(rho), t(dc), gamma=1e-3))
    ref = oflt.sensitivity_filter(rho, dc, dims, r, 1e-3)
    assert rel_max(got, ref) < 1e-13


@pytest.mark.parametrize("dims", [(8, 4, 4), (40, 24, 16)])
def test_oc_update_unfiltered_given_dc(dims):
    from paper_2201_12931_gb300 import Params, TopoGrid
    g = TopoGrid(dims, Params(levels=1))
    x = synth.uniform_field(dims, 53, 0.1, 0.6)
    dc = -synth.uniform_field(dims, 54, 0.01, 5.0)
    xg = t(x)
    ch = g.oc_update_unfiltered(0.2, 0.35, xg, t(dc))
    xo, cho, lam, steps = ooc.oc_update_unfiltered(x, dc, 0.35, 0.2)
    assert np.abs(n(xg) - xo).max() < 1e-7
    assert abs(ch - cho) < 1e-7
