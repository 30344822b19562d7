"""The density filter for callers that cannot allocate GPU memory.

topo_filter_noalloc serves code that must not call cudaMalloc/cudaFree where
it filters (a caching allocator owns the device memory, or the loop must not
stall on the device-wide synchronisation those calls can cause).  It keeps
its scratch in one static device array.  These tests call it through the
C-ABI twice in a row -- a transpose and then a forward filter with another
radius, so the second call reuses scratch the first one left behind -- and
check both results against topo_filter on a handle of the same grid and
against the oracle's filter, at the filter tolerance of the other GPU tests
(1e-14 relative); once on a small ragged grid and once at the documented
limits (1,048,576 elements, radius 6 with its 905 neighbour offsets).
Collected last so that a stop-at-first-failure run has run every other test
first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import filter as oflt

pytestmark = pytest.mark.gpu


def _noalloc(lib, dims, r, x, transpose):
    out = torch.empty_like(x)
    st = lib.topo_filter_noalloc(dims[0], dims[1], dims[2], float(r), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(out.data_ptr()), 1 if transpose else 0,
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.topo_last_error(None).decode()
    return out


def _rel(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("dims,radii", [((33, 17, 9), (2.5, 1.5)), ((128, 128, 64), (6.0, 6.0))])
def test_noalloc_filter_matches_handle_and_oracle_two_calls(dims, radii):
    from paper_2201_12931_gb300 import Params, TopoGrid, _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    g = TopoGrid(dims, Params(levels=1))
    a_np = synth.uniform_field(dims, 61, -1.0, 1.0)
    b_np = synth.uniform_field(dims, 62)
    for x_np, r, tr in ((a_np, radii[0], True), (b_np, radii[1], False)):
        x = torch.tensor(x_np, device=dev)
        got = _noalloc(lib, dims, r, x, tr)
        ref = g.filter(r, x, transpose=tr)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert _rel(got, ref) <= 1e-14
        orc = oflt.density_filter_T(x_np, dims, r) if tr else oflt.density_filter(x_np, dims, r)
        assert _rel(got, orc) <= 1e-14
    g.close()


def test_noalloc_filter_rejects_grids_above_its_scratch():
    """One element over the limit: rejected before any launch, with real
    buffers of that size so that nothing could be written out of bounds."""
    from paper_2201_12931_gb300 import _lib
    lib = _lib.load()
    ne = 128 * 128 * 65
    x = torch.zeros(ne, dtype=torch.float64, device="cuda")
    y = torch.zeros(ne, dtype=torch.float64, device="cuda")
    st = lib.topo_filter_noalloc(128, 128, 65, 1.5, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), 0,
                                 None)
    assert st == 1
    assert "at most 1048576" in lib.topo_last_error(None).decode()
    torch.cuda.synchronize()
    assert not bool(y.any())
