"""Numbering of the structured brick grid (oracle; test infrastructure only).

nx*ny*nz unit elements; element id e = i + nx*(j + ny*k); node id
n = i + (nx+1)*(j + (ny+1)*k); DOF 3*n + c (c = x, y, z).  Element (i, j, k)
has the eight corner nodes (i + a_x, j + a_y, k + a_z), local corner number
a = a_x + 2 a_y + 4 a_z, matching oracle.element.CORNERS.
"""
from __future__ import annotations

import numpy as np


def n_nodes(dims):
    nx, ny, nz = dims
    return (nx + 1) * (ny + 1) * (nz + 1)


def n_elems(dims):
    nx, ny, nz = dims
    return nx * ny * nz


def element_nodes(dims) -> np.ndarray:
    """(nel, 8) global node ids of every element's corners."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    out = np.empty((i.size, 8), dtype=np.int64)
    a = 0
    for az in (0, 1):
        for ay in (0, 1):
            for ax in (0, 1):
                out[:, a] = (i + ax) + (nx + 1) * ((j + ay) + (ny + 1) * (k + az))
                a += 1
    return out


def element_dofs(dims) -> np.ndarray:
    """(nel, 24) global DOF ids in local order 3*a + c."""
    en = element_nodes(dims)
    return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(en.shape[0], 24)


def node_coords(dims) -> np.ndarray:
    """(nnodes, 3) integer coordinates (i, j, k) of every node."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
