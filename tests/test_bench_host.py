"""Host-side logic of bench.py, without a GPU.

* The N > 1 path (replicas, one process per GPU): the barrier and the
  max-over-ranks reduction of the step time, run here as two gloo ranks on
  the CPU; the reference arm runs on rank 0 only and the other ranks return
  without work.
* The reference arm's JSON line on a small sample of the workload.
"""
import argparse
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        worst = bench.max_over_ranks(1.5 + rank, ws)   # per-rank step times 1.5 s and 2.5 s
        args = argparse.Namespace(workload="log2d_n65536", steps=1, warmup=0)
        ref = bench.run_reference(args, ws, rank) if rank != 0 else "skipped"
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"worst": worst, "ref": ref}, f)


def test_replica_path_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    for rank in range(ws):
        r = json.load(open(tmp_path / ("rank%d.json" % rank)))
        assert r["worst"] == 2.5               # every rank reports the slowest rank's time
        if rank != 0:
            assert r["ref"] is None             # the reference arm works on rank 0 only


def test_reference_arm_json_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "CPU_SAMPLE_N", 2048)
    args = argparse.Namespace(workload="log2d_n65536", steps=1, warmup=0)
    out = bench.run_reference(args, 1, 0)
    json.dumps(out)
    assert out["impl"] == "reference" and out["unit"] == "s" and out["value"] > 0
    assert out["higher_is_better"] is False and out["n_gpus"] == 1
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and "N=2048" in cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _prof(**ms_work):
    return {c: {"ms": ms, "work": work, "timed": 10, "launches": 10} for c, (ms, work) in ms_work.items()}


def test_roofline_picks_the_dominant_class_and_its_bound():
    sys.path.insert(0, ROOT)
    import bench
    # panel dominant: FP32 flops on the CUDA cores
    r = bench.roofline(_prof(panel=(50.0, 1.5e10), apply=(5.0, 1e9)))
    assert r["kernel"] == "panel" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bench.FP32_SIMT_TFLOPS)
    assert r["achieved"] == pytest.approx(1.5e10 / 50e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None                       # no capture registered
    # the FP64 H^2 product: FP64 pipe
    r = bench.roofline(_prof(h2_matvec=(20.0, 2.3e10), panel=(1.0, 1e9)))
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_TFLOPS
    # a byte-counted class: HBM
    r = bench.roofline(_prof(apply=(30.0, 6e10), panel=(1.0, 1e9)))
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(6e10 / 30e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # FP32 sparsification kernels are FP32-ALU bound, FP64 ones FP64-bound
    assert bench.roofline(_prof(transform=(9.0, 1e10)), sparsify_fp32=True)["peak"] == pytest.approx(bench.FP32_SIMT_TFLOPS)
    assert bench.roofline(_prof(transform=(9.0, 1e10)), sparsify_fp32=False)["peak"] == bench.FP64_TFLOPS
