"""The density filter for callers that cannot allocate GPU memory.

topo_filter_noalloc serves code that must not call cudaMalloc/cudaFree where
it filters (a caching allocator owns the device memory, or the loop must not
stall on the device-wide synchronisation those calls can cause).  It keeps
its scratch in one static device array.  This test calls it through the
C-ABI twice in a row -- a transpose and then a forward filter with another
radius, so the second call reuses scratch the first one left behind -- and
checks both results against topo_filter on a handle of the same grid, at
the filter tolerance of the other GPU tests (1e-14 relative).  Collected
last so that a stop-at-first-failure run has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, dims, r, x, transpose):
    out = torch.empty_like(x)
    st = lib.topo_filter_noalloc(dims[0], dims[1], dims[2], float(r), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(out.data_ptr()), 1 if transpose else 0,
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.topo_last_error(None).decode()
    return out


def test_noalloc_filter_matches_handle_filter_two_calls():
    from paper_2201_12931_gb300 import Params, TopoGrid, _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    dims = (33, 17, 9)
    g = TopoGrid(dims, Params(levels=1))
    a = torch.tensor(synth.uniform_field(dims, 61, -1.0, 1.0), device=dev)
    b = torch.tensor(synth.uniform_field(dims, 62), device=dev)
    for x, r, tr in ((a, 2.5, True), (b, 1.5, False)):
        got = _noalloc(lib, dims, r, x, tr)
        ref = g.filter(r, x, transpose=tr)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    g.close()


def test_noalloc_filter_rejects_grids_above_its_scratch():
    from paper_2201_12931_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.topo_filter_noalloc(128, 128, 65, 1.5, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr() + 8), 0,
                                 None)
    assert st == 1
    assert "at most 1048576" in lib.topo_last_error(None).decode()
