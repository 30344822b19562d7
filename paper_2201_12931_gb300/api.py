"""Thin Python wrapper over the C-ABI: torch CUDA tensors in, raw pointers out.

PyTorch provides device memory and the stream; all arithmetic runs in the
library's kernels.  Tensors must be contiguous CUDA tensors of the stated
dtype; the wrapper checks shapes and dtypes and raises TopoError on any
non-OK status (solves return TOPO_MAXITER in their result instead).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L


class TopoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


@dataclass
class Params:
    E0: float = 1.0
    Emin: float = 1e-9
    nu: float = 0.3
    penal: float = 3.0
    levels: int = 3
    pre: int = 2
    post: int = 2
    omega: float = 0.35
    precision: int = L.TOPO_FP64
    inner_tol: float = 1e-4
    inner_max_it: int = 500
    max_refine: int = 12
    homogenize: int = 0
    graphs: int = 1
    outer_residual: int = 0
    tensor_cores: int = 0
    cg_check: int = 0

    def to_c(self) -> L.TopoParams:
        p = L.TopoParams()
        for k in self.__dataclass_fields__:
            setattr(p, k, getattr(self, k))
        return p


@dataclass
class SolveResult:
    status: int
    iters: int
    relres: float
    outer_steps: int
    solve_ms: float
    graph_replays: int = 0


def _ptr(t: torch.Tensor, dtype, numel=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class TopoGrid:
    """One structured grid with its solver workspace on the current CUDA device."""

    def __init__(self, dims, params: Params | None = None, stream: torch.cuda.Stream | None = None):
        self.lib = L.load()
        self.dims = tuple(int(d) for d in dims)
        self.params = params or Params()
        nx, ny, nz = self.dims
        self.ne = nx * ny * nz
        self.nn = (nx + 1) * (ny + 1) * (nz + 1)
        self.stream = stream or torch.cuda.current_stream()
        self._h = C.c_void_p()
        cp = self.params.to_c()
        st = self.lib.topo_create_grid(nx, ny, nz, C.byref(cp), C.c_void_p(self.stream.cuda_stream), C.byref(self._h))
        if st != L.TOPO_OK:
            raise TopoError(st, self.lib.topo_last_error(None).decode())
        self.generation = 0

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if self._h:
            self.lib.topo_destroy_grid(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != L.TOPO_OK and st not in allow:
            raise TopoError(st, self.lib.topo_last_error(self._h).decode())
        return st

    def _dev(self):
        return torch.device("cuda", torch.cuda.current_device())

    # -- hot path ----------------------------------------------------------
    def set_density(self, rho: torch.Tensor):
        self._check(self.lib.topo_set_density(self._h, _ptr(rho, torch.float64, self.ne, "rho")))
        self.generation += 1

    def set_bc_loads(self, fixed: torch.Tensor, f: torch.Tensor):
        self._check(self.lib.topo_set_bc_loads(self._h, _ptr(fixed, torch.uint8, 3 * self.nn, "fixed"),
                                               _ptr(f, torch.float64, 3 * self.nn, "f")))
        self.generation += 1

    def solve(self, rel_tol=1e-8, max_it=1000, out: torch.Tensor | None = None, allow_breakdown=False):
        """Returns (u or None, SolveResult).  TOPO_MAXITER is reported, not
        raised; TOPO_BREAKDOWN too with allow_breakdown (the best iterate and
        its residual are returned either way)."""
        it = C.c_int(0)
        rr = C.c_double(0.0)
        up = _ptr(out, torch.float64, 3 * self.nn, "out") if out is not None else None
        st = self.lib.topo_solve_state(self._h, rel_tol, max_it, up, C.byref(it), C.byref(rr))
        self._check(st, allow=(L.TOPO_MAXITER,) + ((L.TOPO_BREAKDOWN,) if allow_breakdown else ()))
        self.generation += 1
        s = self.stats()
        return out, SolveResult(st, it.value, rr.value, s.outer_steps, s.solve_ms, s.graph_replays)

    def compliance_and_sensitivity(self, dc: torch.Tensor | None = None):
        Cv = C.c_double(0.0)
        dp = _ptr(dc, torch.float64, self.ne, "dc") if dc is not None else None
        self._check(self.lib.topo_compliance_and_sensitivity(self._h, C.byref(Cv), dp))
        return Cv.value, dc

    def state_step_host(self, rho: torch.Tensor, rel_tol=1e-8, max_it=1000, dc: torch.Tensor | None = None,
                        allow_breakdown=False):
        """topo_state_step_host: density from host memory, solve, C, and dc
        into a host tensor.  rho and dc are CPU float64 tensors (pinned for
        asynchronous copies).  Returns (C, dc, SolveResult)."""
        for name, v in (("rho", rho), ("dc", dc)):
            if v is None:
                continue
            if not isinstance(v, torch.Tensor) or v.is_cuda or v.dtype != torch.float64 or not v.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CPU float64 tensor")
            if v.numel() != self.ne:
                raise ValueError(f"{name} must have {self.ne} elements, got {v.numel()}")
        Cv = C.c_double(0.0)
        it = C.c_int(0)
        rr = C.c_double(0.0)
        st = self.lib.topo_state_step_host(self._h, C.c_void_p(rho.data_ptr()), float(rel_tol), int(max_it),
                                           C.byref(Cv), C.c_void_p(dc.data_ptr()) if dc is not None else None,
                                           C.byref(it), C.byref(rr))
        self._check(st, allow=(L.TOPO_MAXITER,) + ((L.TOPO_BREAKDOWN,) if allow_breakdown else ()))
        self.generation += 1
        s = self.stats()
        return Cv.value, dc, SolveResult(st, it.value, rr.value, s.outer_steps, s.solve_ms, s.graph_replays)

    def filter(self, r: float, x: torch.Tensor, transpose=False, out: torch.Tensor | None = None):
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.topo_filter(self._h, float(r), _ptr(x, torch.float64, self.ne, "in"),
                                         _ptr(out, torch.float64, self.ne, "out"), 1 if transpose else 0))
        return out

    def oc_update(self, r: float, move: float, volfrac: float, x: torch.Tensor, dc: torch.Tensor) -> float:
        ch = C.c_double(0.0)
        self._check(self.lib.topo_oc_update(self._h, float(r), float(move), float(volfrac),
                                            _ptr(x, torch.float64, self.ne, "x"),
                                            _ptr(dc, torch.float64, self.ne, "dc"), C.byref(ch)))
        return ch.value

    def sensitivity_filter(self, r: float, rho: torch.Tensor, dc: torch.Tensor, gamma: float = 1e-3,
                           out: torch.Tensor | None = None):
        """Eq. sensitivity filter: H(rho dc) / max(gamma, rho)."""
        out = torch.empty_like(dc) if out is None else out
        self._check(self.lib.topo_sensitivity_filter(self._h, float(r), float(gamma),
                                                     _ptr(rho, torch.float64, self.ne, "rho"),
                                                     _ptr(dc, torch.float64, self.ne, "dc"),
                                                     _ptr(out, torch.float64, self.ne, "out")))
        return out

    def oc_update_unfiltered(self, move: float, volfrac: float, x: torch.Tensor, dc: torch.Tensor,
                             passive: torch.Tensor | None = None) -> float:
        """OC step with already filtered sensitivities and the volume of x itself;
        passive (uint8 per element): 0 active, 1 solid, 2 void."""
        ch = C.c_double(0.0)
        pp = None if passive is None else _ptr(passive, torch.uint8, self.ne, "passive")
        self._check(self.lib.topo_oc_update_unfiltered(self._h, float(move), float(volfrac), pp,
                                                       _ptr(x, torch.float64, self.ne, "x"),
                                                       _ptr(dc, torch.float64, self.ne, "dc"), C.byref(ch)))
        return ch.value

    def gravity_load(self, w: float, rho: torch.Tensor, f_ext: torch.Tensor | None = None,
                     out: torch.Tensor | None = None):
        """f_ext + self-weight of density rho (w per unit-density element, -z)."""
        out = torch.empty(3 * self.nn, dtype=torch.float64, device=rho.device) if out is None else out
        fe = None if f_ext is None else _ptr(f_ext, torch.float64, 3 * self.nn, "f_ext")
        self._check(self.lib.topo_gravity_load(self._h, float(w), _ptr(rho, torch.float64, self.ne, "rho"), fe,
                                               _ptr(out, torch.float64, 3 * self.nn, "out")))
        return out

    def gravity_sensitivity(self, w: float, dc: torch.Tensor):
        """dc += load term of the self-weight sensitivity (in place)."""
        self._check(self.lib.topo_gravity_sensitivity(self._h, float(w), _ptr(dc, torch.float64, self.ne, "dc")))
        return dc

    # -- step-level entry points --------------------------------------------
    def level_dims(self, level: int):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.topo_level_dims(self._h, level, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def level_nodes(self, level: int):
        nx, ny, nz = self.level_dims(level)
        return (nx + 1) * (ny + 1) * (nz + 1)

    def apply_operator(self, u, level=0, precision=L.TOPO_FP64):
        y = torch.empty_like(u)
        n = 3 * self.level_nodes(level)
        self._check(self.lib.topo_apply_operator(self._h, level, precision, _ptr(u, torch.float64, n, "u"),
                                                 _ptr(y, torch.float64, n, "y")))
        return y

    def jacobi_sweep(self, u, f, level=0, precision=L.TOPO_FP64):
        y = torch.empty_like(u)
        n = 3 * self.level_nodes(level)
        self._check(self.lib.topo_jacobi_sweep(self._h, level, precision, _ptr(u, torch.float64, n, "u"),
                                               _ptr(f, torch.float64, n, "f"), _ptr(y, torch.float64, n, "out")))
        return y

    def residual(self, u, f, level=0, precision=L.TOPO_FP64):
        y = torch.empty_like(u)
        n = 3 * self.level_nodes(level)
        self._check(self.lib.topo_residual(self._h, level, precision, _ptr(u, torch.float64, n, "u"),
                                           _ptr(f, torch.float64, n, "f"), _ptr(y, torch.float64, n, "r")))
        return y

    def restrict(self, fine, level=0):
        nc = 3 * self.level_nodes(level + 1)
        out = torch.empty(nc, dtype=torch.float64, device=fine.device)
        self._check(self.lib.topo_restrict(self._h, level, _ptr(fine, torch.float64, 3 * self.level_nodes(level)),
                                           _ptr(out, torch.float64, nc)))
        return out

    def prolong_add(self, coarse, fine, level=0):
        self._check(self.lib.topo_prolong_add(self._h, level, _ptr(coarse, torch.float64, 3 * self.level_nodes(level + 1)),
                                              _ptr(fine, torch.float64, 3 * self.level_nodes(level))))
        return fine

    def level_density(self, level: int):
        nx, ny, nz = self.level_dims(level)
        out = torch.empty(nx * ny * nz, dtype=torch.float64, device=self._dev())
        self._check(self.lib.topo_level_density(self._h, level, _ptr(out, torch.float64)))
        return out

    def vcycle(self, r, precision=L.TOPO_FP64):
        z = torch.empty_like(r)
        self._check(self.lib.topo_vcycle(self._h, precision, _ptr(r, torch.float64, 3 * self.nn, "r"),
                                         _ptr(z, torch.float64, 3 * self.nn, "z")))
        return z

    def stats(self) -> L.TopoSolveStats:
        s = L.TopoSolveStats()
        self._check(self.lib.topo_get_stats(self._h, C.byref(s)))
        return s

    def reset_solution(self):
        self._check(self.lib.topo_reset_solution(self._h))

    def profile_enable(self, on=True):
        self._check(self.lib.topo_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, mode: int):
        """(launches, total_ms) per kernel precision [fp64, fp32, fp32 with BF16
        iterates, double-fp32, fp32 with tensor-core element products] for
        operator kind `mode`."""
        n = (C.c_longlong * 5)()
        ms = (C.c_double * 5)()
        self._check(self.lib.topo_profile_read(self._h, mode, n, ms))
        return list(n), list(ms)

    def launch_count(self) -> int:
        v = C.c_longlong(0)
        self._check(self.lib.topo_launch_count(self._h, C.byref(v)))
        return v.value


def measure_peak(kind: int, stream=None):
    """Measured arithmetic peak of the CUDA cores (topo_measure_peak):
    kind 0 = FP64 FMA, 1 = FP32 FMA, 2 = paired FP32 FMA.  Returns
    (TFLOP/s, launch ms)."""
    lib = L.load()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    st = lib.topo_measure_peak(kind, C.c_void_p(s), C.byref(tf), C.byref(ms))
    if st != L.TOPO_OK:
        raise TopoError(st, lib.topo_last_error(None).decode())
    return tf.value, ms.value
