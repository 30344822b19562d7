"""Host-side checks of the C-ABI library (no GPU needed).

The library builds for sm_103a, loads, exports every entry point that
include/topo.h declares, and validates arguments before any CUDA call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_12931_gb300 import build as b
    from paper_2201_12931_gb300 import _lib
    b.build()
    return _lib.load()


def _declared():
    with open(os.path.join(ROOT, "include", "topo.h")) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"^\s*(?:topo_status|const char\*)\s+(topo_\w+)\s*\(", src, re.M)))


def test_header_and_binding_agree():
    from paper_2201_12931_gb300 import _lib
    assert set(_declared()) == set(_lib.exported_names())


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_params(lib):
    from paper_2201_12931_gb300._lib import TopoParams
    p = TopoParams()
    assert lib.topo_default_params(C.byref(p)) == 0
    assert (p.E0, p.Emin, p.nu, p.penal, p.omega, p.pre, p.post) == (1.0, 1e-9, 0.3, 3.0, 0.35, 2, 2)
    assert p.homogenize == 0
    assert lib.topo_default_params(None) == 1


@pytest.mark.parametrize("dims,levels,msg", [
    ((0, 4, 4), 1, "positive"),
    ((6, 4, 4), 3, "divisible"),
    ((6, 4, 4), 0, "levels"),
    ((896, 896, 896), 1, "too large"),     # 3 * 897^3 nodal entries >= 2^31
])
def test_create_grid_rejects_bad_arguments(lib, dims, levels, msg):
    from paper_2201_12931_gb300._lib import TopoParams
    p = TopoParams()
    lib.topo_default_params(C.byref(p))
    p.levels = levels
    h = C.c_void_p()
    st = lib.topo_create_grid(*dims, C.byref(p), None, C.byref(h))
    assert st == 1
    assert not h
    assert msg in lib.topo_last_error(None).decode()


def test_create_grid_rejects_bad_omega_and_nu(lib):
    from paper_2201_12931_gb300._lib import TopoParams
    p = TopoParams()
    lib.topo_default_params(C.byref(p))
    p.levels = 1
    p.omega = 1.5
    h = C.c_void_p()
    assert lib.topo_create_grid(2, 2, 2, C.byref(p), None, C.byref(h)) == 1
    lib.topo_default_params(C.byref(p))
    p.levels = 1
    p.nu = 0.5
    assert lib.topo_create_grid(2, 2, 2, C.byref(p), None, C.byref(h)) == 1
    lib.topo_default_params(C.byref(p))
    p.levels = 1
    p.homogenize = 3
    assert lib.topo_create_grid(2, 2, 2, C.byref(p), None, C.byref(h)) == 1
    assert "homogenize" in lib.topo_last_error(None).decode()
    lib.topo_default_params(C.byref(p))
    p.levels = 1
    p.homogenize = 2
    p.precision = 2
    assert lib.topo_create_grid(2, 2, 2, C.byref(p), None, C.byref(h)) == 1


def test_null_handle_calls_are_rejected(lib):
    assert lib.topo_destroy_grid(None) == 1
    assert lib.topo_set_density(None, None) == 1
    assert lib.topo_solve_state(None, 1e-8, 10, None, None, None) == 1
    assert lib.topo_filter(None, 1.5, None, None, 0) == 1
    assert lib.topo_oc_update(None, 1.5, 0.2, 0.3, None, None, None) == 1
    assert lib.topo_sensitivity_filter(None, 1.5, 1e-3, None, None, None) == 1
    assert lib.topo_oc_update_unfiltered(None, 0.2, 0.3, None, None, None, None) == 1
    assert lib.topo_gravity_load(None, 0.1, None, None, None) == 1
    assert lib.topo_gravity_sensitivity(None, 0.1, None) == 1
    assert lib.topo_compliance_and_sensitivity(None, None, None) == 1
    assert lib.topo_state_step_host(None, None, 1e-8, 10, None, None, None, None) == 1
    assert lib.topo_vcycle(None, 0, None, None) == 1


def test_params_struct_matches_header(lib):
    """Every field of topo_params in the header is in the ctypes mirror, in order."""
    import re
    from paper_2201_12931_gb300._lib import TopoParams, TopoSolveStats
    hdr = open(os.path.join(ROOT, "include", "topo.h")).read()

    def fields(struct):
        body = re.search(r"typedef struct \{([^{}]*)\} " + struct + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                names += [v.strip() for v in decl.split(None, 1)[1].split(",")]
        return names
    assert fields("topo_params") == [f[0] for f in TopoParams._fields_]
    assert fields("topo_solve_stats") == [f[0] for f in TopoSolveStats._fields_]


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2201_12931_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
