"""Seeded synthetic inputs shared by the oracle-side and the CUDA-side tests.

This module holds problem data only -- random density fields, Dirichlet
masks and nodal load vectors -- and none of the method's arithmetic (no
stiffness, no filter, no solver). Both the CPU oracle and the CUDA path are
fed from here, so that a parity test compares the two on identical inputs.

Conventions (shared with the C-ABI in include/topo.h):
  * grid of nx*ny*nz unit hex8 elements, element id e = i + nx*(j + ny*k);
  * (nx+1)*(ny+1)*(nz+1) nodes, node id n = i + (nx+1)*(j + (ny+1)*k);
  * 3 DOFs per node, node-major: dof = 3*n + c with c = 0,1,2 for x,y,z;
  * z is the vertical axis.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the e-th draw of stream `seed` mixes seed + (e+1)*golden_gamma.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Return draws start..start+count-1 of the splitmix64 stream `seed` (uint64)."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """53-bit doubles in [0, 1) from the top bits of splitmix64 draws."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform01_at(seed: int, idx) -> np.ndarray:
    """Draws number idx (any array of indices) of stream `seed`: the same
    values uniform01(seed, n)[idx] gives, without generating the others."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_field(dims, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Per-element field U[lo, hi) in element order (x fastest), float64."""
    nx, ny, nz = dims
    return lo + (hi - lo) * uniform01(seed, nx * ny * nz)


def sample_without_replacement(seed: int, n: int, k: int) -> np.ndarray:
    """k distinct indices in [0, n) drawn from stream `seed` (rejection of repeats)."""
    out: list[int] = []
    seen: set[int] = set()
    start = 0
    while len(out) < k:
        draws = uniform01(seed, 4 * k, start)
        start += 4 * k
        for v in draws:
            i = int(v * n)
            if i not in seen:
                seen.add(i)
                out.append(i)
                if len(out) == k:
                    break
    return np.asarray(out, dtype=np.int64)


def n_nodes(dims) -> int:
    nx, ny, nz = dims
    return (nx + 1) * (ny + 1) * (nz + 1)


def node_index(dims, i, j, k):
    nx, ny, _ = dims
    return np.asarray(i) + (nx + 1) * (np.asarray(j) + (ny + 1) * np.asarray(k))


def _line_weights(npts: int) -> np.ndarray:
    """Consistent nodal loads of a unit-intensity line load over unit segments."""
    w = np.ones(npts)
    if npts > 1:
        w[0] = w[-1] = 0.5
    return w


@dataclass
class Problem:
    """Boundary conditions and loads of one synthetic workload."""
    dims: tuple
    fixed: np.ndarray          # uint8, 3*nodes, 1 = Dirichlet (u = 0)
    f: np.ndarray              # float64, 3*nodes
    name: str = ""
    info: dict = field(default_factory=dict)


def cantilever_fixed_at(dims, dofs) -> np.ndarray:
    """Dirichlet flags of the cantilever (face x = 0 clamped) at given DOFs."""
    nx, _, _ = dims
    node = np.asarray(dofs) // 3
    return (node % (nx + 1) == 0).astype(np.uint8)


def cantilever(dims) -> Problem:
    """Cantilever: face x=0 clamped; unit -z line load along the bottom edge
    (i = nx, all j, k = 0), consistent nodal weights (ends 1/2)."""
    nx, ny, nz = dims
    nn = n_nodes(dims)
    fixed = np.zeros(3 * nn, dtype=np.uint8)
    jj, kk = np.meshgrid(np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    clamp = node_index(dims, 0, jj.ravel(), kk.ravel())
    for c in range(3):
        fixed[3 * clamp + c] = 1
    f = np.zeros(3 * nn)
    edge = node_index(dims, nx, np.arange(ny + 1), 0)
    f[3 * edge + 2] = -_line_weights(ny + 1)
    return Problem(tuple(dims), fixed, f, name=f"cantilever_{nx}x{ny}x{nz}")


def mbb_half(dims) -> Problem:
    """MBB half-beam: symmetry u_x = 0 on face x=0; roller u_z = 0 on the bottom
    far line (i = nx, all j, k = 0); u_y = 0 at node (nx, 0, 0) to remove the
    free y-translation; unit -z line load on the top line at the symmetry plane
    (i = 0, all j, k = nz), consistent nodal weights."""
    nx, ny, nz = dims
    nn = n_nodes(dims)
    fixed = np.zeros(3 * nn, dtype=np.uint8)
    jj, kk = np.meshgrid(np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    face = node_index(dims, 0, jj.ravel(), kk.ravel())
    fixed[3 * face + 0] = 1
    roller = node_index(dims, nx, np.arange(ny + 1), 0)
    fixed[3 * roller + 2] = 1
    fixed[3 * node_index(dims, nx, 0, 0) + 1] = 1
    f = np.zeros(3 * nn)
    top = node_index(dims, 0, np.arange(ny + 1), nz)
    f[3 * top + 2] = -_line_weights(ny + 1)
    return Problem(tuple(dims), fixed, f, name=f"mbb_{nx}x{ny}x{nz}")


def arch_bridge(dims, deck_layers, slot_halfwidth, q=1.0) -> Problem:
    """Bridge-like domain with non-design regions (Sec. 5, Example 2; the
    geometry is only in the paper's figures, so this is a stand-in): the top
    `deck_layers` element layers are passive solid; the elements within
    slot_halfwidth of mid-span in the lower half of the height are passive
    void; supports on the two bottom end lines (u_z = 0 on (0, j, 0) and
    (nx, j, 0), u_x = 0 on (0, j, 0), u_y = 0 at (0, 0, 0)); uniform pressure q
    on the top surface, consistent nodal loads q/4 per adjacent unit face.
    info["passive"]: uint8 per element, 0 active, 1 solid, 2 void."""
    nx, ny, nz = dims
    nn = n_nodes(dims)
    fixed = np.zeros(3 * nn, dtype=np.uint8)
    left = node_index(dims, 0, np.arange(ny + 1), 0)
    right = node_index(dims, nx, np.arange(ny + 1), 0)
    fixed[3 * left + 2] = 1
    fixed[3 * right + 2] = 1
    fixed[3 * left + 0] = 1
    fixed[3 * node_index(dims, 0, 0, 0) + 1] = 1
    f = np.zeros(3 * nn)
    wx, wy = _line_weights(nx + 1), _line_weights(ny + 1)
    jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    top = node_index(dims, ii.ravel(), jj.ravel(), nz)
    f[3 * top + 2] = -q * np.outer(wy, wx).ravel()
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    passive = np.zeros(nx * ny * nz, dtype=np.uint8)
    passive[(k >= nz - deck_layers).ravel()] = 1
    slot = (np.abs(i + 0.5 - nx / 2) <= slot_halfwidth) & (k < nz // 2)
    passive[slot.ravel()] = 2
    return Problem(tuple(dims), fixed, f, name=f"arch_bridge_{nx}x{ny}x{nz}", info=dict(passive=passive))


# ---------------------------------------------------------------------------
# Named workloads.  Each one records the grid, material, solver levels and the
# recipe of its density field.  Density recipes that need the density filter
# (a step of the method) are stated here as data; each side applies its own
# filter implementation to the raw field returned by raw_density().
# ---------------------------------------------------------------------------

MATERIAL = dict(E0=1.0, Emin=1e-9, nu=0.3, penal=3.0)

WORKLOADS = {
    "cantilever_48x24x24_fp64_oc20": dict(
        dims=(48, 24, 24), problem="cantilever", levels=3, precision="fp64",
        density=dict(kind="const", value=0.3), rel_tol=1e-8,
        oc=dict(iters=20, rmin=1.5, move=0.2, volfrac=0.3)),
    "cantilever_128x64x64_mixed": dict(
        dims=(128, 64, 64), problem="cantilever", levels=5, precision="mixed",
        density=dict(kind="uniform_filtered", seed=1, lo=1e-3, hi=1.0, rmin=1.5),
        rel_tol=1e-8),
    "mbb_96x48x48_grad": dict(
        dims=(96, 48, 48), problem="mbb", levels=4, precision="fp64",
        density=dict(kind="uniform_filtered", seed=2, lo=0.05, hi=1.0, rmin=2.0),
        rel_tol=1e-12, fd=dict(h=1e-4, count=64, seed=2)),
    "cantilever_256x128x128_oc50": dict(
        dims=(256, 128, 128), problem="cantilever", levels=5, precision="mixed_bf16",
        density=dict(kind="const", value=0.12), rel_tol=1e-8,
        oc=dict(iters=50, rmin=2.5, move=0.2, volfrac=0.12)),
    # the cantilever cases of the paper's timing table (Sec. 5, Example 1):
    # grid and iteration count from the table; volume fraction, filter
    # radius and move limit are not stated there (TOP3D125-style defaults)
    "cantilever_64x32x32_oc64": dict(
        dims=(64, 32, 32), problem="cantilever", levels=4, precision="mixed",
        density=dict(kind="const", value=0.12), rel_tol=1e-8,
        oc=dict(iters=64, rmin=1.5, move=0.2, volfrac=0.12)),
    "cantilever_128x64x64_oc49": dict(
        dims=(128, 64, 64), problem="cantilever", levels=5, precision="mixed",
        density=dict(kind="const", value=0.12), rel_tol=1e-8,
        oc=dict(iters=49, rmin=1.5, move=0.2, volfrac=0.12)),
    # bridge stand-ins with non-design regions (Sec. 5, Examples 2 and 4):
    # 140 x 10 x 20 domain at 448 x 32 x 64, deck 1.5 (5 layers) passive
    # solid, void slot (the 4 elements within 1.5 of mid-span, lower half),
    # volume fraction 0.14 of the active region; the gravity variant adds
    # the self-weight load
    "arch_bridge_448x32x64_passive": dict(
        dims=(448, 32, 64), problem="arch_bridge", levels=5, precision="mixed",
        density=dict(kind="const", value=0.14), rel_tol=1e-8,
        bridge=dict(deck_layers=5, slot_halfwidth=1.5, q=1.0, weight=0.0),
        oc=dict(iters=30, rmin=1.5, move=0.2, volfrac=0.14)),
    "arch_bridge_448x32x64_gravity": dict(
        dims=(448, 32, 64), problem="arch_bridge", levels=5, precision="mixed",
        density=dict(kind="const", value=0.14), rel_tol=1e-8,
        bridge=dict(deck_layers=5, slot_halfwidth=1.5, q=1.0, weight=0.05),
        oc=dict(iters=30, rmin=1.5, move=0.2, volfrac=0.14)),
    # the foot-bridge size of the paper's Example 4 (1152 x 64 x 256, 49
    # iterations, self-weight with non-design regions) on the bridge
    # stand-in geometry (deck 20 layers, slot at mid-span)
    "footbridge_1152x64x256_gravity": dict(
        dims=(1152, 64, 256), problem="arch_bridge", levels=6, precision="mixed",
        density=dict(kind="const", value=0.125), rel_tol=1e-8,
        bridge=dict(deck_layers=20, slot_halfwidth=4.5, q=1.0, weight=0.05),
        oc=dict(iters=49, rmin=1.5, move=0.2, volfrac=0.125)),
    "cantilever_768x384x384_mixed": dict(
        dims=(768, 384, 384), problem="cantilever", levels=7, precision="mixed",
        density=dict(kind="uniform_filtered_clipped", seed=3, lo=0.0, hi=1.0,
                     rmin=3.0, clip=(1e-3, 1.0)),
        compliance_tol=1e-6),
}


def make_problem(name: str, dims=None) -> Problem:
    w = WORKLOADS[name]
    dims = tuple(dims or w["dims"])
    if w["problem"] == "arch_bridge":
        b = w["bridge"]
        p = arch_bridge(dims, b["deck_layers"], b["slot_halfwidth"], b["q"])
        p.info.update(w)
        return p
    p = cantilever(dims) if w["problem"] == "cantilever" else mbb_half(dims)
    p.info = dict(w)
    return p


def raw_density(name: str, dims=None) -> np.ndarray:
    """The unfiltered per-element field of a workload's density recipe."""
    w = WORKLOADS[name]
    dims = tuple(dims or w["dims"])
    d = w["density"]
    nel = dims[0] * dims[1] * dims[2]
    if d["kind"] == "const":
        x = np.full(nel, d["value"])
        if w["problem"] == "arch_bridge":   # passive regions start at their values
            pas = make_problem(name, dims).info["passive"]
            x[pas == 1], x[pas == 2] = 1.0, 0.0
        return x
    return uniform_field(dims, d["seed"], d["lo"], d["hi"])
