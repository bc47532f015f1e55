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
        args = argparse.Namespace(workload="log2d_n65536", steps=1, warmup=0, factor="auto")
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
    from paper_1705_04601_gb300 import synth
    real = synth.make_workload
    # the "full" instance of this test: N = 4096 (its structure only scales the sample's phases)
    monkeypatch.setattr(synth, "make_workload", lambda name, n=None, **kw: real(name, n=n or 4096))
    args = argparse.Namespace(workload="log2d_n65536", steps=1, warmup=0, factor="auto")
    out = bench.run_reference(args, 1, 0)
    json.dumps(out)
    assert out["impl"] == "reference" and out["unit"] == "s" and out["value"] > 0
    assert out["higher_is_better"] is False and out["n_gpus"] == 1
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and "N=2048" in cb["sample"]
    assert out["config"]["n"] == 4096 and out["config"]["sample_n"] == 2048 and "N=4096" in cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _prof(**ms_work):
    return {c: {"ms": ms, "work": work, "timed": 10, "launches": 10} for c, (ms, work) in ms_work.items()}


FMA = {"fp64": 1.2, "fp32": 75.0}  # stand-ins for the measured FMA rates


def test_roofline_picks_the_dominant_class_and_its_bound(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6782.4, "bf16_tflops": 1922.5,
                                                          "bf16_tflops_sustained": 1693.4})
    # the tensor-core trailing update: FP32 flops against the three-pass TF32 ceiling
    r = bench.roofline(_prof(gemm_update=(40.0, 4e12), panel=(5.0, 1e9)), FMA)
    assert r["kernel"] == "gemm_update" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(1693.4 * 0.5 / 3.0)
    assert r["achieved"] == pytest.approx(4e12 / 40e-3 / 1e12)
    assert r["tf32_pipe_frac"] == pytest.approx(3.0 * r["achieved"] / (1693.4 * 0.5))
    # with CUDA-core updates the same class is FP32 ALU work
    r = bench.roofline(_prof(gemm_update=(40.0, 4e12)), FMA, fp32_gemm_tc=False)
    assert r["bound"] == "alu" and r["peak"] == FMA["fp32"]
    # panel dominant: FP32 flops on the CUDA cores, measured peak
    r = bench.roofline(_prof(panel=(50.0, 1.5e10), apply=(5.0, 1e9)), FMA)
    assert r["kernel"] == "panel" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == FMA["fp32"] and "measured" in r["peak_source"]
    assert r["achieved"] == pytest.approx(1.5e10 / 50e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None                       # no capture registered
    # the FP64 H^2 product: FP64 pipe
    r = bench.roofline(_prof(h2_matvec=(20.0, 2.3e10), panel=(1.0, 1e9)), FMA)
    assert r["bound"] == "alu" and r["peak"] == FMA["fp64"]
    # a byte-counted class: HBM
    r = bench.roofline(_prof(apply=(30.0, 6e10), panel=(1.0, 1e9)), FMA)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6782.4
    assert r["achieved"] == pytest.approx(6e10 / 30e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # FP32 sparsification kernels are FP32-ALU bound, FP64 ones FP64-bound
    assert bench.roofline(_prof(transform=(9.0, 1e10)), FMA, sparsify_fp32=True)["peak"] == FMA["fp32"]
    assert bench.roofline(_prof(transform=(9.0, 1e10)), FMA, sparsify_fp32=False)["peak"] == FMA["fp64"]


def test_cpu_baseline_scaling_counts_agree_with_the_planner():
    """The work counts that scale the oracle sample (the oracle's own schedule,
    predicted pattern and symbolic factorization) equal the library
    planner's factor flops, and the Cholesky's are half the LU's."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1705_04601_gb300 import h2sp as H
    from paper_1705_04601_gb300 import synth
    h, _ = synth.make_workload("inv3d_sphere_n262144", n=4096)
    st = H.h2sp_query(H.h2sp_analyze(H.H2Input(h, device=None)))
    _, f_lu, e_lu = bench._oracle_work(h, "lu")
    _, f_ch, e_ch = bench._oracle_work(h, "chol")
    assert f_lu == pytest.approx(st["factor_flops"], rel=1e-12)
    assert f_ch == pytest.approx(st["chol_flops"], rel=1e-12) and f_ch == pytest.approx(0.5 * f_lu, rel=1e-12)
    assert e_lu == e_ch > 0
    assert bench._work_ratios(h, h, "chol") == pytest.approx((1.0, 1.0, 1.0))


_FAKED_RUN = r'''
import argparse
import json
import sys
import types

import numpy as np
import torch

sys.path.insert(0, sys.argv[1])
import bench  # noqa: E402
from paper_1705_04601_gb300 import build, synth  # noqa: E402
from paper_1705_04601_gb300 import h2sp as H  # noqa: E402

build.build = lambda: None
_real_make = synth.make_workload
synth.make_workload = lambda name, n=None, **kw: _real_make(name, n=2048)


class Ev:
    def record(self, s=None):
        pass

    def elapsed_time(self, o):
        return 10.0


torch.cuda.Event = lambda enable_timing=True: Ev()
torch.cuda.synchronize = lambda *a, **k: None
torch.cuda.current_device = lambda: 0
torch.Tensor.cuda = lambda self, *a, **k: self
torch.Tensor.pin_memory = lambda self, *a, **k: self


class FakeHandle:
    def close(self):
        pass


class FakeInput:
    def __init__(self, h, device="cuda", nonblocking_from=None, host=None):
        self.h = h


classes = H.KERNEL_CLASSES
H.H2Input = FakeInput
H.h2sp_analyze = lambda inp: FakeHandle()
H.h2sp_sparsify_analyzed = lambda an, inp, stream=None, flags=0: FakeHandle()
H.h2sp_factor = lambda hd, prec, stream=None: None
RES = float(sys.argv[2])
H.h2sp_solve = lambda hd, b, x, mode=0, tol=1e-10, maxit=50, restart=30, stream=None: types.SimpleNamespace(
    iters=5, rel_residual=RES, status=0 if RES <= 1e-10 else -6)
H.h2sp_profile = lambda hd, timing=-1, reset=False: {
    c: {"launches": 3, "timed": 3, "ms": (5.0 if c == "panel" else 1.0), "work": 1e9} for c in classes}
H.h2sp_query = lambda hd: {"factor_flops": 3e12, "chol_flops": 1.5e12, "max_front": 100, "nsupernodes": 3,
                           "nnz": 1000, "front_elems": 10000}
H.h2sp_measure_peak = lambda kind, stream=None: 1.2 if kind == 0 else 75.0
H.h2sp_solve_host = lambda an, inp, bp, ldb, xp, ldx, nrhs, **kw: types.SimpleNamespace(
    iters=5, rel_residual=5e-11, status=0)
torch.cuda.current_stream = lambda *a, **k: types.SimpleNamespace(cuda_stream=0)
H.h2sp_apply = lambda hd, op, x, y, stream=None: y.copy_(x)

args = argparse.Namespace(gpus=1, steps=2, warmup=1, impl="ours", workload="log2d_n65536", fp64_steps=1,
                          e2e_steps=2, factor="auto", sparsify_prec="fp32", solver="gmres", no_e2e=False,
                          no_cpu_baseline=True, tune="auto", no_construct=True)
out = bench.run_ours(args, 1, 0, 0)
print(json.dumps(out))
'''


def _faked(tmp_path, res):
    import subprocess
    src = tmp_path / "faked_run.py"
    src.write_text(_FAKED_RUN)
    r = subprocess.run([sys.executable, str(src), ROOT, repr(res)], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bench_value_is_null_when_a_step_does_not_converge(tmp_path):
    """A mixed step that stops above 1e-10 (ENOCONV) publishes no time and no speed-up."""
    out = _faked(tmp_path, 5e-10)
    assert out["converged"] is False and out["value"] is None and out["speedup_mixed_vs_fp64"] is None


def test_bench_json_line_with_faked_library(tmp_path):
    """bench.run_ours end to end on the CPU, with the library calls and the
    CUDA events faked (a child process, so the fakes stay there): the JSON
    line carries every field of the measurement contract."""
    import subprocess
    src = tmp_path / "faked_run.py"
    src.write_text(_FAKED_RUN)
    r = subprocess.run([sys.executable, str(src), ROOT, "5e-11"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks", "gpu_launches",
              "cpu_baseline", "factor_gflops_fp32", "factor_gflops_fp64"):
        assert k in out, k
    assert out["higher_is_better"] is False and out["steps"] == 2 and out["warmup"] == 1
    assert out["config"]["workload"] == "log2d_n65536"
    assert out["roofline"]["kernel"] == "panel" and out["roofline"]["frac"] > 0
    assert set(out["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert out["e2e"]["entry"] == "h2sp_solve_host" and out["e2e"]["value"] is not None
    assert out["factor_gflops_fp64"] > 0 and out["gpu_launches"] > 0
    assert out["converged"] is True and out["value"] is not None and out["config"]["factor"] == "block LU"
    assert out["fma_peaks_tflops"] == {"fp64": 1.2, "fp32": 75.0}


def test_tune_cache_roundtrip(tmp_path, monkeypatch):
    """The autotuner's store: keyed by device and structure sizes; the
    environment's cache file is read before the shipped one and written."""
    sys.path.insert(0, ROOT)
    from paper_1705_04601_gb300 import tune as T
    st = {"n": 262144, "nsupernodes": 66, "max_front": 89578, "chol_flops": 3.7e14}
    k = T.key(st, "NVIDIA GB300")
    assert k == T.key(dict(st), "NVIDIA GB300") and k != T.key(dict(st, max_front=1), "NVIDIA GB300")
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("H2SP_TUNE_CACHE", str(cache))
    assert T.load(k) is None
    sched = {"tiles_per_cta": 16, "panel_sms": 8, "lookahead": 1}
    T.store(k, sched, 123.0)
    assert T.load(k) == sched
    assert json.load(open(cache))[k]["factor_ms"] == 123.0
    assert set(T.DEFAULT) == set(T.CANDIDATES) and all(T.DEFAULT[n] in T.CANDIDATES[n] for n in T.DEFAULT)


def test_tune_descent_finds_the_coordinate_optimum():
    """The tuner's search on a fake timer: with a separable cost it reaches
    the best value of every knob, trying each other value once per knob; a
    gain inside the noise margin does not move it off the defaults."""
    sys.path.insert(0, ROOT)
    from paper_1705_04601_gb300 import tune as T
    cands = {"a": [0, 1, 2], "b": [5, 6], "c": [1, 0]}
    best = {"a": 2, "b": 6, "c": 0}
    calls = []

    def cost(s):
        calls.append(dict(s))
        return 100.0 + sum(10.0 * abs(s[k] - best[k]) for k in s)

    sched, ms = T.descend(cost, {"a": 0, "b": 5, "c": 1}, cands)
    assert sched == best and ms == 100.0
    assert len(calls) == 1 + sum(len(v) - 1 for v in cands.values())
    # every candidate changes one knob of a schedule timed before it
    assert all(any(sum(c[k] != d[k] for k in c) == 1 for d in calls[:i]) for i, c in enumerate(calls) if i)
    flat = lambda s: 100.0 - (0.5 if s["a"] == 1 else 0.0)  # 0.5 % better: inside the 1 % margin
    assert T.descend(flat, {"a": 0, "b": 5, "c": 1}, cands)[0] == {"a": 0, "b": 5, "c": 1}
    assert T.descend(lambda s: 100.0 - (5.0 if s["a"] == 1 else 0.0), {"a": 0, "b": 5, "c": 1},
                     cands)[0] == {"a": 1, "b": 5, "c": 1}


def test_shipped_schedules_are_candidates():
    """Every schedule stored in the shipped tuned.json sets each knob of the
    tuner, to one of its candidate values, under a well-formed key."""
    sys.path.insert(0, ROOT)
    from paper_1705_04601_gb300 import tune as T
    d = json.load(open(T.SHIPPED))
    assert d
    for k, v in d.items():
        dev, *sizes = k.split("|")
        assert dev and [s.split("=")[0] for s in sizes] == ["n", "sn", "front", "chol"]
        assert set(v["schedule"]) == set(T.CANDIDATES)
        assert all(v["schedule"][name] in T.CANDIDATES[name] for name in T.CANDIDATES)
        assert v["factor_ms"] > 0
