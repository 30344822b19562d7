"""GB300 (sm_103a) homogenized-multigrid topology-optimisation hot path.

The CUDA library libtopo_gb300.so (built in-tree from csrc/) implements the
C-ABI of include/topo.h; this package is its thin Python binding.
"""
from . import _lib
from ._lib import TOPO_DF32, TOPO_FP32_TC, TOPO_FP64, TOPO_MIXED, TOPO_MIXED_BF16, TOPO_OK, TOPO_MAXITER
from .api import Params, SolveResult, TopoError, TopoGrid

__all__ = ["TopoGrid", "Params", "SolveResult", "TopoError", "TOPO_DF32", "TOPO_FP32_TC", "TOPO_FP64", "TOPO_MIXED", "TOPO_MIXED_BF16",
           "TOPO_OK", "TOPO_MAXITER"]
