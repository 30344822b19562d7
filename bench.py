#!/usr/bin/env python
"""Benchmark of the homogenized-MGPCG topology-optimisation hot path on GB300.

One step = one pass of the whole hot path over the synthetic workload:
set_density (homogenized levels + coarsest factorisation), state solve from
u = 0 (mixed precision: FP32 inner MGPCG inside FP64 refinement), compliance +
sensitivity, filter transpose + OC update.  The metric is the state-solve time
in seconds (lower is better); the compliance of the mixed solve is checked
against an all-FP64 GPU solve of the same grid to 1e-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--dims NXxNYxNZ] [--fp64-ref full|skip]
                  [--cpu-baseline on|off]

Under torchrun (N > 1) every rank solves its own replica of the workload
(the solve needs no data from other ranks); timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "cantilever_768x384x384_mixed"
CPU_SAMPLE_DIMS = (96, 48, 48)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--dims", default=None, help="override grid, e.g. 96x48x48")
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--rel-tol", type=float, default=1e-6,
                    help="relative residual of the timed (mixed) solve")
    ap.add_argument("--fp64-tol", type=float, default=1e-6,
                    help="relative residual of the timed all-FP64 comparison solve")
    ap.add_argument("--fp64-ref", choices=["full", "skip"], default="full")
    ap.add_argument("--cpu-baseline", choices=["on", "off"], default="on")
    ap.add_argument("--coarsening", choices=["density", "modulus", "galerkin"], default="density",
                    help="coarse operators: SIMP of the mean child density (Sec. 4.2.2), mean child modulus, "
                         "or stored Galerkin element matrices")
    ap.add_argument("--filter", choices=["density", "sensitivity"], default="density",
                    help="OC loop: density filter (chain rule) or the paper's sensitivity filter")
    ap.add_argument("--graphs", choices=["on", "off"], default="on",
                    help="replay PCG iterations from captured CUDA graphs (off: direct launches)")
    ap.add_argument("--oc-iters", type=int, default=0, help="OC loop: iterations (default: the workload's)")
    ap.add_argument("--cg-check", choices=["batched", "every"], default="batched",
                    help="host reads of r.r: after batches sized from the contraction rate, or every CG iteration")
    ap.add_argument("--sweeps", default="2,2", help="Jacobi sweeps before,after the coarse correction")
    ap.add_argument("--tensor-cores", choices=["off", "on"], default="off",
                    help="FP32 operators with tcgen05 element products instead of the modal kernel")
    ap.add_argument("--oc-fp64", choices=["on", "off"], default="on",
                    help="OC loop: also run the all-FP64 loop for the drift comparison")
    ap.add_argument("--oc-loop", action="store_true",
                    help="run the workload's topology-optimisation loop (mixed and FP64) instead of the step bench")
    ap.add_argument("--oracle-table", choices=["on", "off"], default="on",
                    help="time the oracle and the GPU path on the small configurations (C1-C3) in the same run")
    ap.add_argument("--traffic-from", default=None,
                    help="write profiles/traffic.json from an ncu CSV of dram__bytes_{read,write}.sum of the "
                         "operator kernels of a run with --dims (see profiles/traffic.json for the command)")
    ap.add_argument("--traffic-command", default="", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload(args):
    import synth
    w = dict(synth.WORKLOADS[args.workload])
    dims = tuple(int(v) for v in args.dims.split("x")) if args.dims else tuple(w["dims"])
    levels = args.levels or w["levels"]
    while levels > 1 and any(d % (1 << (levels - 1)) for d in dims):
        levels -= 1
    return w, dims, levels


def physical_density(grid, name, dims, dev):
    """The workload's density recipe on the device (filtering with the
    library's own filter kernel)."""
    import torch
    import synth
    d = synth.WORKLOADS[name]["density"]
    raw = torch.tensor(synth.raw_density(name, dims), device=dev)
    if d["kind"] == "const":
        return raw
    rho = grid.filter(d["rmin"], raw)
    if "clip" in d:
        rho.clamp_(d["clip"][0], d["clip"][1])
    return rho


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on the host's cores, on a bounded sample
# ---------------------------------------------------------------------------

def host_threads():
    """Cores this process may run on (the oracle's thread budget)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _cpu_seconds():
    import resource
    r = resource.getrusage(resource.RUSAGE_SELF)
    return r.ru_utime + r.ru_stime


def oracle_env():
    n = str(host_threads())
    return dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)

def cpu_sample(name, dims, rel_tol):
    """Oracle state solve of the workload recipe at `dims`; returns seconds."""
    import numpy as np
    import synth
    from oracle import filter as oflt, state as ostate
    w = synth.WORKLOADS[name]
    pb = synth.make_problem(name, dims)
    raw = synth.raw_density(name, dims)
    d = w["density"]
    rho = raw if d["kind"] == "const" else oflt.density_filter(raw, dims, d["rmin"])
    if "clip" in d:
        rho = np.clip(rho, *d["clip"])
    t0 = time.perf_counter()
    u, info = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=rel_tol, method="mgpcg", return_info=True)
    return time.perf_counter() - t0, info


def run_cpu_child(args):
    w, dims, _ = workload(args)
    sample = CPU_SAMPLE_DIMS
    times = []
    c0, t0 = _cpu_seconds(), time.perf_counter()
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            c0, t0 = _cpu_seconds(), time.perf_counter()
        t, info = cpu_sample(args.workload, sample, args.rel_tol)
        if i >= args.warmup:
            times.append(t)
    util = (_cpu_seconds() - c0) / max(time.perf_counter() - t0, 1e-9)
    print(json.dumps({"times": times, "sample_dims": sample, "iters": info["iters"], "cpu_util": util}))


def cpu_baseline(args, steps=3, warmup=1):
    """Spawns the oracle in a fresh process allowed all host cores; one
    untimed solve, then `steps` timed ones of the bounded sample, scaled to
    the workload by element count (multigrid work is linear in it)."""
    cores = host_threads()
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-child", "--workload", args.workload,
           "--steps", str(steps), "--warmup", str(warmup), "--rel-tol", str(args.rel_tol)]
    if args.dims:
        cmd += ["--dims", args.dims]
    out = subprocess.run(cmd, capture_output=True, text=True, env=oracle_env(), timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    _, dims, _ = workload(args)
    ne_full = dims[0] * dims[1] * dims[2]
    s = res["sample_dims"]
    scale = ne_full / (s[0] * s[1] * s[2])
    t = statistics.mean(res["times"])
    return {
        "value": t * scale,
        "unit": "s",
        "cores": cores,
        "kind": "oracle",
        "extrapolated": True,
        "scale_factor": round(scale, 3),
        "sample_s": round(t, 4),
        "cpu_utilisation": round(res["cpu_util"], 2),
        "sample": (f"oracle FP64 state solve (assembled CSR K, Galerkin-MG PCG to rel. residual {args.rel_tol:g}, "
                   f"{res['iters']} it) of the same recipe on a {s[0]}x{s[1]}x{s[2]} grid, mean of {steps} after "
                   f"{warmup} untimed, {cores} threads allowed: {t:.2f} s, extrapolated by element count "
                   f"x{scale:.0f} to {dims[0]}x{dims[1]}x{dims[2]}"),
    }


# the small configurations both the oracle and the GPU path run in full
ORACLE_TABLE = (
    ("C1", "cantilever_48x24x24_fp64_oc20", "s per OC iteration (density filter, solve to 1e-8, sensitivity, OC)"),
    ("C2", "cantilever_128x64x64_mixed", "s per state solve to rel. residual 1e-8 from u = 0"),
    ("C3", "mbb_96x48x48_grad", "s per compliance gradient (filter, solve to 1e-10, sensitivity, filter transpose)"),
)


def run_oracle_child(label):
    """One configuration of ORACLE_TABLE on the oracle, timed in this process."""
    import synth
    from oracle import filter as oflt, state as ostate
    _, name, _ = next(c for c in ORACLE_TABLE if c[0] == label)
    w = synth.WORKLOADS[name]
    dims = tuple(w["dims"])
    pb = synth.make_problem(name)
    x = synth.raw_density(name)
    c0, t0 = _cpu_seconds(), time.perf_counter()
    if label == "C1":
        oc = w["oc"]
        ostate.oc_iteration(dims, x, pb.fixed, pb.f, oc["rmin"], oc["volfrac"], oc["move"], tol=w["rel_tol"])
        detail = "1 iteration from x = 0.3"
    elif label == "C2":
        rho = oflt.density_filter(x, dims, w["density"]["rmin"])
        c0, t0 = _cpu_seconds(), time.perf_counter()     # the input filter is not part of the solve
        _, info = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-8, method="mgpcg", return_info=True)
        detail = f"Galerkin-MG PCG, {info['iters']} it"
    else:
        rmin = w["density"]["rmin"]
        rho = oflt.density_filter(x, dims, rmin)
        u = ostate.solve_state(dims, rho, pb.fixed, pb.f, tol=1e-10, method="mgpcg")
        _, _, dc = ostate.compliance_and_sensitivity(dims, rho, u, pb.f)
        oflt.density_filter_T(dc, dims, rmin)
        detail = "Galerkin-MG PCG"
    wall = time.perf_counter() - t0
    print(json.dumps({"s": wall, "cpu_util": (_cpu_seconds() - c0) / max(wall, 1e-9), "detail": detail}))


def oracle_time(label):
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", label]
    out = subprocess.run(cmd, capture_output=True, text=True, env=oracle_env(), timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def gpu_time(label, dev):
    """The same configuration on the GPU path: CUDA-event time, median of 3
    after one untimed repetition (C1: mean over the 20-iteration loop)."""
    import torch
    import synth
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_FP64, TOPO_MIXED
    from paper_2201_12931_gb300.autograd import compliance
    _, name, _ = next(c for c in ORACLE_TABLE if c[0] == label)
    w = synth.WORKLOADS[name]
    dims = tuple(w["dims"])
    pb = synth.make_problem(name)
    prec = TOPO_FP64 if w["precision"] == "fp64" else TOPO_MIXED
    g = TopoGrid(dims, Params(levels=w["levels"], precision=prec))
    g.set_bc_loads(torch.tensor(pb.fixed, device=dev), torch.tensor(pb.f, device=dev))
    x0 = torch.tensor(synth.raw_density(name), device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    times = []
    if label == "C1":
        oc = w["oc"]
        x = x0.clone()
        dc = torch.empty(g.ne, dtype=torch.float64, device=dev)
        for _ in range(oc["iters"]):
            a, b = ev(), ev()
            a.record()
            g.set_density(g.filter(oc["rmin"], x))
            g.solve(w["rel_tol"], 20000)
            g.compliance_and_sensitivity(dc)
            g.oc_update(oc["rmin"], oc["move"], oc["volfrac"], x, dc)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
        t = statistics.mean(times[1:])
        detail = f"mean of iterations 2-{oc['iters']} of the loop, {w['precision']}"
    else:
        rmin = w["density"]["rmin"]
        for i in range(4):
            a, b = ev(), ev()
            if label == "C2":
                g.set_density(g.filter(rmin, x0))
                g.reset_solution()
                a.record()
                g.solve(1e-8, 20000)
                b.record()
            else:
                xr = x0.clone().requires_grad_(True)
                g.reset_solution()
                a.record()
                compliance(xr, g, rmin, rel_tol=1e-10).backward()
                b.record()
            torch.cuda.synchronize()
            if i > 0:
                times.append(a.elapsed_time(b) / 1e3)
        t = statistics.median(times)
        detail = f"median of 3 after one untimed, {w['precision']}"
    g.close()
    return t, detail


def oracle_table(dev):
    rows = []
    for label, name, unit in ORACLE_TABLE:
        o = oracle_time(label)
        tg, dg = gpu_time(label, dev)
        rows.append({"config": label, "workload": name, "unit": unit, "oracle_s": round(o["s"], 4),
                     "oracle_detail": o["detail"], "oracle_cores": host_threads(),
                     "oracle_cpu_utilisation": round(o["cpu_util"], 2), "gpu_s": round(tg, 5), "gpu_detail": dg,
                     "oracle_over_gpu": round(o["s"] / tg, 1)})
    return rows


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


OP_NAMES = {0: "K.u", 1: "Jacobi sweep", 2: "residual", 3: "first Jacobi sweep",
            4: "K.p with p = z + beta p fused", 5: "first two Jacobi sweeps fused"}
PREC_NAMES = ("fp64", "fp32", "fp32, bf16 iterates", "double-fp32", "fp32, tensor-core element products")


def op_bytes(mode, prec, nn, ne):
    """Algorithmic HBM bytes of one fine-level operator launch: the nodal
    vectors it must read and write (3 DOFs per node) plus one modulus per
    element; s = 8 (FP64 kernel) or 4 (FP32 kernel)."""
    if prec == 3:   # double-FP32 arithmetic on FP64 u, f, E; residual written as FP32, K.u as FP64
        return 3 * nn * ({0: 8 + 8, 2: 8 + 8 + 4}[mode]) + ne * 8
    if prec == 2:   # BF16 iterates u (in) and u' (out, FP32 for the last sweep), FP32 f and residual
        su, sf, so = 2, 4, 2
        return 3 * nn * ({0: su + so, 1: su + sf + so, 2: su + sf + 4, 3: sf + so, 4: 4 * 4, 5: sf + so}[mode]) + ne * 4
    s = 8 if prec == 0 else 4   # prec 1 and 4: FP32 vectors
    # K.u: u, y | Jacobi: u, f, u' | residual: u, f, r | first: f, u' | K.p fused: z, p_old, q, p |
    # first two sweeps: f, u''
    nvec = {0: 2, 1: 3, 2: 3, 3: 2, 4: 4, 5: 2}[mode]
    return nvec * 3 * nn * s + ne * s


def kernel_table(grid, nn, ne):
    peak, src = peaks()
    rows = []
    for mode in range(6):
        cnt, ms = grid.profile_read(mode)
        for prec in (0, 1, 2, 3, 4):
            if not cnt[prec]:
                continue
            b = op_bytes(mode, prec, nn, ne)
            avg = ms[prec] / cnt[prec]
            gbs = b / (avg / 1e3) / 1e9
            rows.append({"kernel": f"{OP_NAMES[mode]} ({PREC_NAMES[prec]}) fine level",
                         "mode": mode, "prec": prec, "launches": cnt[prec], "total_ms": round(ms[prec], 3),
                         "avg_launch_ms": round(avg, 4), "algorithmic_bytes_per_launch": b,
                         "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
    return rows, peak, src


KERNEL_SOURCES = ["paper_2201_12931_gb300/csrc/stencil.cu", "paper_2201_12931_gb300/csrc/operator.cuh",
                  "paper_2201_12931_gb300/csrc/opio.cuh", "paper_2201_12931_gb300/csrc/dfloat.cuh",
                  "paper_2201_12931_gb300/csrc/tc_op.cu"]


def kernel_kind(name):
    """(mode, prec) of an operator kernel from its demangled ncu name, else None:
    k_op<T, TU, TO, MODE, DOT> (T float / double / dfl, TU bf16 for BF16
    iterates) and k_op_tc<MODE, DOT>."""
    import re
    m = re.search(r"k_op_tc<(?:\(int\))?(\d), (?:\(bool\))?(\d)>", name)
    if m:
        return int(m.group(1)), 4
    m = re.search(r"k_op<([^,]+), ([^,]+), ([^,]+), (?:\(int\))?(\d), (?:\(bool\))?(\d)>", name)
    if not m:
        return None
    t, tu = m.group(1).strip(), m.group(2).strip()
    prec = 3 if "dfl" in t else (0 if t == "double" else (2 if "bfloat16" in tu else 1))
    return int(m.group(4)), prec


def write_traffic(args):
    """Fine-level launches (largest grid of each kind) of an ncu CSV with
    dram__bytes_read.sum / dram__bytes_write.sum -> profiles/traffic.json."""
    import csv
    _, dims, _ = workload(args)
    launches = {}
    with open(args.traffic_from) as fh:
        rows = [r for r in csv.reader(fh) if len(r) > 10]
    hdr = rows[0]
    ix = {k: hdr.index(k) for k in ("ID", "Kernel Name", "Grid Size", "Metric Name", "Metric Unit", "Metric Value")}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1, "usecond": 1e3, "msecond": 1e6}
    for r in rows[1:]:
        kind = kernel_kind(r[ix["Kernel Name"]])
        if kind is None:
            continue
        d = launches.setdefault(r[ix["ID"]], {"kind": kind, "grid": r[ix["Grid Size"]], "name": r[ix["Kernel Name"]]})
        d[r[ix["Metric Name"]]] = float(r[ix["Metric Value"]].replace(",", "")) * scale.get(r[ix["Metric Unit"]], 1)
    def volume(g):
        return eval(g.replace("(", "").replace(")", "").replace(",", "*"))
    best = {}
    for d in launches.values():
        if "dram__bytes_read.sum" not in d:
            continue
        k = d["kind"]
        if k not in best or volume(d["grid"]) > volume(best[k]["grid"]):
            best[k] = d
    entries = [{"mode": k[0], "prec": k[1], "kernel": d["name"].split("(")[0].replace("void ", "")[:120],
                "dims": list(dims), "grid": d["grid"], "dram_bytes_read": int(d["dram__bytes_read.sum"]),
                "dram_bytes_write": int(d["dram__bytes_write.sum"]),
                "duration_ns": int(d.get("gpu__time_duration.sum", 0))} for k, d in sorted(best.items())]
    out = {"kernel_sha256": kernel_hash(), "command": args.traffic_command,
           "note": (f"first fine-level launch (largest grid) of each operator kernel kind on the {dims[0]}x{dims[1]}x"
                    f"{dims[2]} grid; bench.py scales the bytes to the workload by element count (the operator "
                    "kernels stream the fine-level vectors once per launch, so traffic grows with the elements); "
                    "durations are cold-cache and serialised under ncu"),
           "entries": entries}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(mode, prec, ne):
    """DRAM bytes per launch of an operator kernel from profiles/traffic.json,
    scaled to `ne` elements; None if absent or taken on other kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("kernel_sha256") != kernel_hash():
        return None
    for e in t.get("entries", []):
        if e["mode"] == mode and e["prec"] == prec:
            d = e["dims"]
            return (e["dram_bytes_read"] + e["dram_bytes_write"]) * ne / (d[0] * d[1] * d[2])
    return None


_ALU = {}


def alu_peaks():
    """FP64 / FP32 FMA peaks of this GPU in TFLOP/s, measured once per process
    with the library's own microbenchmark (topo_measure_peak)."""
    if not _ALU:
        from paper_2201_12931_gb300.api import measure_peak
        for kind, name in ((0, "fp64"), (1, "fp32"), (2, "fp32x2")):
            tf, ms = measure_peak(kind)
            _ALU[name] = round(tf, 3)
            _ALU[name + "_ms"] = round(ms, 4)
    return _ALU
# algorithmic FP64 flops of one element in the modal operator (FMA = 2):
# in-plane transform of the new face 24, z butterfly 21, modulus scaling 8,
# modal block stiffness 33, inverse z butterfly 21, face accumulation 12,
# inverse in-plane transform 24, corner sums and residual 12
MODAL_FLOPS_PER_ELEMENT = 24 + 21 + 8 + 33 + 21 + 12 + 24 + 12
# FP32 flops of one element of the double-FP32 residual: the same operator as
# 133 pair additions (TwoSum of the high words + two low-word adds = 8 flops)
# and 34 pair products (one multiply and three FMAs = 7 flops)
DF_FLOPS_PER_ELEMENT = 133 * 8 + 34 * 7


def roofline_entry(r, peak, src, ne):
    if r["prec"] in (0, 3):   # FP64 / double-FP32 operators: bound by the arithmetic pipes, not by HBM
        alu = alu_peaks()
        fl = (MODAL_FLOPS_PER_ELEMENT if r["prec"] == 0 else DF_FLOPS_PER_ELEMENT) * ne
        pk = alu["fp64"] if r["prec"] == 0 else max(alu["fp32"], alu["fp32x2"])
        tflops = fl / (r["avg_launch_ms"] / 1e3) / 1e12
        tr = measured_traffic(r["mode"], r["prec"], ne)
        return {"bound": "alu", "achieved": round(tflops, 4), "peak": pk, "unit": "TFLOP/s",
                "frac": round(tflops / pk, 4), "traffic": None if tr is None else int(tr), "kernel": r["kernel"],
                "launches": r["launches"], "avg_launch_ms": r["avg_launch_ms"],
                "algorithmic_flops_per_launch": fl,
                "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"],
                "achieved_gbs": r["achieved_gbs"],
                "peak_source": "measured: topo_measure_peak " + ("FP64" if r["prec"] == 0 else "FP32")
                               + " FMA chains, this GPU, this run"}
    tr = measured_traffic(r["mode"], r["prec"], ne)
    return {"bound": "hbm", "achieved": r["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": r["frac"],
            "traffic": None if tr is None else int(tr), "kernel": r["kernel"], "launches": r["launches"],
            "avg_launch_ms": r["avg_launch_ms"], "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"],
            "peak_source": src}


def roofline(rows, peak, src, ne):
    """Dominant fine-level operator kernel (largest total time) from the live event records."""
    if not rows:
        return None
    return roofline_entry(max(rows, key=lambda v: v["total_ms"]), peak, src, ne)


def ku_roofline(rows, peak, src, ne):
    """The FP32 K.u kernel of the metric (HBM-bound form), whatever its share."""
    r = [v for v in rows if v["mode"] in (0, 4) and v["prec"] in (1, 4)]
    return roofline_entry(r[0], peak, src, ne) if r else None


COARSENING = {"density": 0, "modulus": 1, "galerkin": 2}


def max_over_ranks(vals, dev=None):
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (the replicas' times); the list itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_FP64, TOPO_MIXED, TOPO_MIXED_BF16, TOPO_OK

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w, dims, levels = workload(args)
    prec = {"fp64": TOPO_FP64, "mixed": TOPO_MIXED, "mixed_bf16": TOPO_MIXED_BF16}[w["precision"]]
    nx, ny, nz = dims
    ne, nn = nx * ny * nz, (nx + 1) * (ny + 1) * (nz + 1)
    pb = synth.make_problem(args.workload, dims)
    fixed_d = torch.tensor(pb.fixed, device=dev)
    f_d = torch.tensor(pb.f, device=dev)
    del pb
    rmin = w.get("oc", {}).get("rmin", w["density"].get("rmin", 1.5))
    move = w.get("oc", {}).get("move", 0.2)

    hom = COARSENING[args.coarsening]
    pre, post = (int(v) for v in args.sweeps.split(","))
    g = TopoGrid(dims, Params(levels=levels, precision=prec, homogenize=hom, graphs=int(args.graphs == "on"),
                              cg_check=int(args.cg_check == "every"), tensor_cores=int(args.tensor_cores == "on"),
                              pre=pre, post=post))
    rho0 = physical_density(g, args.workload, dims, dev)
    volfrac = w.get("oc", {}).get("volfrac", float(rho0.mean()))
    g.set_bc_loads(fixed_d, f_d)
    dc = torch.empty(ne, dtype=torch.float64, device=dev)
    xw = torch.empty(ne, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step(record):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.set_density(rho0)
        g.reset_solution()
        _, res = g.solve(args.rel_tol, 20000)
        e1.record(stream)
        C, _ = g.compliance_and_sensitivity(dc)
        xw.copy_(rho0)
        ch = g.oc_update(rmin, move, volfrac, xw, dc)
        e2.record(stream)
        if record is not None:
            record.append((e0, e1, e2, res, C, ch))
        return res, C

    for _ in range(args.warmup):
        step(None)
    rec = []
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = g.launch_count()
    sampler.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(rec)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t0
    clocks = sampler.stop()
    launches = g.launch_count() - launches0
    if world > 1:
        dist.barrier()
    # per-kernel device times: the same steps again with CUDA events around
    # every fine-level operator launch (direct launches instead of the CUDA
    # graphs of the timed steps, whose kernels are the same)
    g.profile_enable(True)
    for _ in range(args.steps):
        step(None)
    torch.cuda.synchronize()
    g.profile_enable(False)
    solve_s = [a.elapsed_time(b) / 1e3 for a, b, _, _, _, _ in rec]
    step_s = [a.elapsed_time(c) / 1e3 for a, _, c, _, _, _ in rec]
    rows, peak, src = kernel_table(g, nn, ne)
    roof = roofline(rows, peak, src, ne)
    roof_ku = ku_roofline(rows, peak, src, ne)
    res_last, C_mixed = rec[-1][3], rec[-1][4]
    t_solve = statistics.mean(solve_s)
    t_step = statistics.mean(step_s)
    t_solve, t_step = max_over_ranks([t_solve, t_step], dev)

    # end to end through one C-ABI call with host buffers (topo_state_step_host):
    # H2D of the step's density from pinned memory, moduli and coarse levels,
    # the solve from u = 0, C and dc, D2H of dc (and of C)
    host_rho = rho0.cpu().pin_memory()
    host_dc = torch.empty(ne, dtype=torch.float64).pin_memory()
    e2e = []
    for i in range(args.steps):
        g.reset_solution()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        Cv, _, _ = g.state_step_host(host_rho, args.rel_tol, 20000, dc=host_dc)
        e2e.append(time.perf_counter() - t1)

    out = {
        "metric": "state-solve s & K·u HBM GB/s at 113M hex; mixed vs FP64 GPU at 1e-6 compliance",
        "value": round(t_solve, 5),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_step * 1e3, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64" if prec != TOPO_FP64 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload if not args.dims else f"{args.workload}@{nx}x{ny}x{nz}",
                   "grid": f"{nx}x{ny}x{nz}", "elements": ne, "dofs": 3 * nn, "levels": levels,
                   "rel_tol": args.rel_tol, "precision": w["precision"], "coarsening": args.coarsening,
                   "sweeps": args.sweeps,
                   "l2": "inputs larger than L2 (fine-level vectors >= 129 MB)" if 12 * nn > 129e6
                   else "inputs smaller than L2 (no flush)"},
        "solve": {"status": res_last.status, "inner_iters": res_last.iters, "outer_steps": res_last.outer_steps,
                  "relres_fp64": res_last.relres, "compliance": C_mixed,
                  "solve_s_per_step": [round(v, 5) for v in solve_s]},
        "gpu_launches": launches,
        "wall_s_timed": round(t_wall, 3),
        "e2e": {"value": round(statistics.mean(e2e), 5), "unit": "s",
                "h2d_bytes_per_step": ne * 8, "d2h_bytes_per_step": ne * 8 + 8,
                "call": "topo_state_step_host (density in, solve from u = 0, C and dc out; pinned host buffers)"},
        "roofline": roof,
        "roofline_ku": roof_ku,
        "operator_kernels": rows,
        "kernel_timing": (f"CUDA events on the handle's stream around every fine-level operator launch of "
                          f"{args.steps} further steps of the same workload right after the timed ones "
                          "(direct launches; the timed steps replay CUDA graphs of the same kernels)"),
        "alu_peaks_tflops": alu_peaks(),
        "clocks": clocks,
    }
    if args.fp64_ref == "full" and prec != TOPO_FP64:
        g64 = TopoGrid(dims, Params(levels=levels, precision=TOPO_FP64, homogenize=hom,
                                    graphs=int(args.graphs == "on")))
        g64.set_bc_loads(fixed_d, f_d)
        g64.set_density(rho0)
        # timed like the mixed arm: untimed warm-up solve, then CUDA events
        # around solves from u = 0 (CUDA graphs on, no launch profiling)
        g64.solve(args.fp64_tol, 20000)
        t64s = []
        for _ in range(3):
            g64.reset_solution()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, r64 = g64.solve(args.fp64_tol, 20000)
            b.record(stream)
            torch.cuda.synchronize()
            t64s.append(a.elapsed_time(b) / 1e3)
        t64 = statistics.median(t64s)
        C64_tol, _ = g64.compliance_and_sensitivity()
        _, r64b = g64.solve(1e-10, 20000)      # warm-started from the solution at fp64_tol
        C_ref, _ = g64.compliance_and_sensitivity()
        out["fp64_gpu"] = {"solve_s": round(t64, 4), "solve_s_all": [round(v, 4) for v in t64s],
                           "timing": "median of 3 solves from u = 0 after one untimed, CUDA events, "
                                     "CUDA graphs on as in the mixed arm",
                           "rel_tol": args.fp64_tol, "iters": r64.iters,
                           "status": r64.status, "compliance_rel_err": abs(C64_tol - C_ref) / abs(C_ref),
                           "compliance_at_tol": C64_tol, "reference_compliance_1e-10": C_ref,
                           "reference": "FP64 solve to 1e-10 warm-started from the fp64_tol solution",
                           "reference_status": r64b.status, "reference_iters": r64b.iters}
        out["compliance_rel_err_mixed_vs_fp64_ref"] = abs(C_mixed - C_ref) / abs(C_ref)
        out["mixed_speedup_vs_fp64"] = round(t64 / t_solve, 3)
        g64.close()
    if rank == 0 and args.cpu_baseline == "on":
        try:
            out["cpu_baseline"] = cpu_baseline(args)
        except Exception as e:   # the bench line must still print
            out["cpu_baseline"] = {"error": str(e)[-300:]}
    if rank == 0 and world == 1 and args.oracle_table == "on":
        try:
            out["oracle_configs"] = oracle_table(dev)
        except Exception as e:
            out["oracle_configs"] = {"error": str(e)[-300:]}
    g.close()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_oc_loop(args):
    """Algorithm 4 with the density filter for the workload's iteration count,
    once with the workload's precision and once all-FP64 (warm-started solves,
    rel. residual from the workload); prints one JSON line with the time per
    iteration of both and the compliance drift of the first against the second."""
    import torch
    import synth
    from paper_2201_12931_gb300 import Params, TopoGrid, TOPO_FP64, TOPO_MIXED, TOPO_MIXED_BF16
    name = args.workload if "oc" in synth.WORKLOADS[args.workload] else "cantilever_256x128x128_oc50"
    w = synth.WORKLOADS[name]
    dims = tuple(int(v) for v in args.dims.split("x")) if args.dims else tuple(w["dims"])
    levels = args.levels or w["levels"]
    while levels > 1 and any(d % (1 << (levels - 1)) for d in dims):
        levels -= 1
    oc = w["oc"]
    dev = torch.device("cuda", 0)
    pb = synth.make_problem(name, dims)
    fixed_d, f_d = torch.tensor(pb.fixed, device=dev), torch.tensor(pb.f, device=dev)
    ne = dims[0] * dims[1] * dims[2]
    x0 = torch.tensor(synth.raw_density(name, dims), device=dev)
    prec = {"fp64": TOPO_FP64, "mixed": TOPO_MIXED, "mixed_bf16": TOPO_MIXED_BF16}[w["precision"]]
    plabel = w["precision"]
    if prec == TOPO_MIXED_BF16 and args.coarsening == "galerkin":   # stored Galerkin levels run FP32 iterates
        prec, plabel = TOPO_MIXED, "mixed"
    tol = w.get("rel_tol", 1e-8)
    out = {"mode": "oc_loop", "workload": name, "grid": "x".join(map(str, dims)), "levels": levels,
           "rel_tol": tol, "graphs": args.graphs, "cg_check": args.cg_check, "rmin": oc["rmin"], "move": oc["move"],
           "volfrac": oc["volfrac"], "coarsening": args.coarsening, "filter": args.filter}
    bridge = w.get("bridge")
    flt = "sensitivity" if bridge else args.filter     # non-design regions: the paper's scheme
    pas_d = torch.tensor(pb.info["passive"], device=dev) if bridge else None
    weight = bridge["weight"] if bridge else 0.0
    out["filter"] = flt
    if bridge:
        out["self_weight"] = weight
    iters = args.oc_iters or oc["iters"]
    out["iterations"] = iters
    runs = {}
    for label, p in (("mixed", prec), ("fp64", TOPO_FP64))[:2 if args.oc_fp64 == "on" else 1]:
        g = TopoGrid(dims, Params(levels=levels, precision=p, homogenize=COARSENING[args.coarsening],
                                  graphs=int(args.graphs == "on"), cg_check=int(args.cg_check == "every"),
                                  tensor_cores=int(args.tensor_cores == "on")))
        g.set_bc_loads(fixed_d, f_d)
        x = x0.clone()
        dc = torch.empty(ne, dtype=torch.float64, device=dev)
        Cs, its, ms = [], [], []
        for it in range(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if bridge:   # passive deck and slot, pressure + self-weight, sensitivity filter
                g.set_density(x)
                if weight > 0.0:
                    g.set_bc_loads(fixed_d, g.gravity_load(weight, x, f_d))
                _, res = g.solve(tol, 20000)
                C, _ = g.compliance_and_sensitivity(dc)
                if weight > 0.0:
                    g.gravity_sensitivity(weight, dc)
                g.oc_update_unfiltered(oc["move"], oc["volfrac"], x, g.sensitivity_filter(oc["rmin"], x, dc),
                                       passive=pas_d)
            elif flt == "density":
                g.set_density(g.filter(oc["rmin"], x))
                _, res = g.solve(tol, 20000)
                C, _ = g.compliance_and_sensitivity(dc)
                g.oc_update(oc["rmin"], oc["move"], oc["volfrac"], x, dc)
            else:   # the paper's loop: design = physical density, filtered sensitivities
                g.set_density(x)
                _, res = g.solve(tol, 20000)
                C, _ = g.compliance_and_sensitivity(dc)
                g.oc_update_unfiltered(oc["move"], oc["volfrac"], x, g.sensitivity_filter(oc["rmin"], x, dc))
            e1.record()
            torch.cuda.synchronize()
            Cs.append(C)
            its.append(res.iters)
            ms.append(e0.elapsed_time(e1))
        g.close()
        runs[label] = dict(C=Cs, iters=its, ms=ms)
        out[label] = {"ms_per_iteration": round(statistics.mean(ms), 3), "total_s": round(sum(ms) / 1e3, 3),
                      "pcg_iterations": its, "compliance_first": Cs[0], "compliance_last": Cs[-1],
                      "precision": label if label == "fp64" else plabel}
    if "fp64" in runs:
        drift = [abs(a - b) / abs(b) for a, b in zip(runs["mixed"]["C"], runs["fp64"]["C"])]
        out["compliance_drift_max"] = max(drift)
        out["compliance_drift_last"] = drift[-1]
        out["compliance_drift"] = [float(f"{d:.3e}") for d in drift]
    print(json.dumps(out))


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, dims, levels = workload(args)
    cb = cpu_baseline(args, steps=args.steps, warmup=args.warmup)
    print(json.dumps({
        "impl": "reference",
        "metric": "state-solve s & K·u HBM GB/s at 113M hex; mixed vs FP64 GPU at 1e-6 compliance",
        "value": cb["value"], "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": "x".join(map(str, dims)), "levels": levels,
                   "rel_tol": args.rel_tol},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse_args()
    if args.traffic_from:
        write_traffic(args)
    elif args.cpu_child:
        run_cpu_child(args)
    elif args.oracle_child:
        run_oracle_child(args.oracle_child)
    elif args.oc_loop:
        run_oc_loop(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
