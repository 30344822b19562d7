"""Host logic of the multi-rank bench path (replicas only: every rank solves
its own copy of the workload; the only cross-rank step is the maximum of the
timings).  Two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 0.5]


def test_max_over_ranks_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks([3, 4.5]) == [3.0, 4.5]


def test_reference_arm_prints_on_rank0_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle timed on the host) runs on
    rank 0 only; the other ranks return without work or output.  The oracle
    timing itself is replaced by a stub here; its JSON line keeps the
    contract's keys."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    stub = {"value": 1.5, "unit": "s", "cores": 1, "kind": "oracle", "sample": "stub"}
    monkeypatch.setattr(bench, "cpu_baseline", lambda args, steps=1, warmup=0: dict(stub))
    args = bench.parse_args(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 1.5
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"] == {"value": 1.5, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["higher_is_better"] is False and line["steps"] == 2 and line["warmup"] == 3


def test_roofline_entries():
    """The bench line's roofline objects: HBM-bound FP32 kernels against the
    measured copy bandwidth, the FP64 and double-FP32 residuals against the
    measured FP64 / FP32 FMA peaks (stand-in values here: no GPU)."""
    sys.path.insert(0, ROOT)
    import bench
    bench._ALU.update(fp64=1.1, fp32=61.0, fp32x2=63.0)
    ne = 1000
    r32 = {"mode": 0, "prec": 1, "kernel": "K.u (fp32) fine level", "launches": 3, "avg_launch_ms": 0.5,
           "algorithmic_bytes_per_launch": 2e9, "achieved_gbs": 4000.0, "frac": 0.6}
    e = bench.roofline_entry(r32, 6700.0, "measured", ne)
    assert e["bound"] == "hbm" and e["unit"] == "GB/s" and e["peak"] == 6700.0 and e["frac"] == 0.6
    r64 = {"mode": 2, "prec": 0, "kernel": "residual (fp64) fine level", "launches": 2, "avg_launch_ms": 1.0,
           "algorithmic_bytes_per_launch": 1e9, "achieved_gbs": 1000.0, "frac": 0.15}
    e = bench.roofline_entry(r64, 6700.0, "measured", ne)
    tflops = bench.MODAL_FLOPS_PER_ELEMENT * ne / 1e-3 / 1e12
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s" and e["traffic"] is None
    assert abs(e["achieved"] - round(tflops, 4)) < 1e-9
    assert e["peak"] == 1.1 and e["peak_source"].startswith("measured")
    rdf = {"mode": 2, "prec": 3, "kernel": "residual (double-fp32) fine level", "launches": 2, "avg_launch_ms": 0.5,
           "algorithmic_bytes_per_launch": 1e9, "achieved_gbs": 2000.0, "frac": 0.3}
    e = bench.roofline_entry(rdf, 6700.0, "measured", ne)
    assert e["bound"] == "alu" and e["peak"] == 63.0
    assert abs(e["achieved"] - round(bench.DF_FLOPS_PER_ELEMENT * ne / 0.5e-3 / 1e12, 4)) < 1e-9
    # the dominant kernel is the one with the largest total time
    rows = [dict(r32, total_ms=1.5), dict(r64, total_ms=2.0)]
    assert bench.roofline(rows, 6700.0, "measured", ne)["bound"] == "alu"
    assert bench.ku_roofline(rows, 6700.0, "measured", ne)["bound"] == "hbm"
    # BF16-iterate kernels count 2-byte iterates
    nn = 100
    assert bench.op_bytes(1, 2, nn, ne) == 3 * nn * (2 + 4 + 2) + 4 * ne
    assert bench.op_bytes(1, 1, nn, ne) == 3 * 3 * nn * 4 + 4 * ne
    assert bench.op_bytes(2, 3, nn, ne) == 3 * nn * (8 + 8 + 4) + 8 * ne


def test_bench_defaults_follow_the_contract():
    """Defaults: one GPU, at least 3 warm-up steps, a few timed steps, the
    113M-element workload, the oracle as the reference arm."""
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and 1 <= a.steps <= 10
    assert a.impl == "ours" and a.workload == "cantilever_768x384x384_mixed"
    assert a.cpu_baseline == "on" and a.fp64_ref == "full" and a.graphs == "on"
    r = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "4", "--warmup", "3"])
    assert r.impl == "reference" and r.gpus == 2 and r.steps == 4
