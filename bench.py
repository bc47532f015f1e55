#!/usr/bin/env python
"""Time to solution of A x = b at relative residual 1e-10 on one GB300.

One step = the whole hot path on the 2D log-kernel H^2 matrix with 65,536
points (leaf <= 64, basis tolerance 1e-6, 16 right-hand sides): the numeric
sparsification h2sp_sparsify_analyzed (A = U S V^T), h2sp_factor (block LU
of S) and h2sp_solve.  The host analysis of the structure (h2sp_analyze:
level schedule, block pattern of S, symbolic factorization) runs once per
structure, before the timed steps, and is reported as ``analysis_ms``.  Two
paths:

* mixed (the headline): S from FP32 sandwich products (the Householder
  completions stay FP64; --sparsify-prec fp64 keeps them all FP64), FP32
  factorization of S, then restarted GMRES (or iterative refinement,
  --solver ir) on the FP64 H^2 product, preconditioned by FP32 U^T, S^-1 and
  V, until max_k ||b_k - A x_k|| / ||b_k|| <= 1e-10;
* fp64: FP64 sparsification and factorization of S, refinement on the FP64
  H^2 residual to 1e-10 (reported beside it).

Inputs are resident in HBM when the timed region starts (the close blocks are
443 MB, larger than the 129 MB L2, so no flush is needed); ``e2e`` repeats the
mixed step from pinned host buffers with the copies inside the timed region.

``--impl reference`` times the CPU FP64 oracle instead (the reference arm):
each step runs the oracle's full pipeline on a bounded sample.
Under torchrun every rank solves an independent replica; rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solution at rel. residual 1e-10 (s), mixed vs FP64 GPU; factor GFLOP/s"
CPU_SAMPLE_N = 16384

# Nominal peaks, used where MEASURED_PEAKS.json has no entry:
#   FP32 SIMT  = 152 SMs x 128 lanes x 2 flop x 2.070 GHz
#   FP64       = 1.25 TFLOP/s (GB300 nominal)
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_TFLOPS = 1.25

# DRAM traffic of the dominant kernel from an ncu capture: per kernel class,
# dram bytes read + written over the class's algorithmic work in the captured
# run, valid while the kernel's source file is unchanged (sha256 prefix of
# "src").  The bench's traffic figure is this ratio times the class's average
# work per launch.  Empty: the current captures (profiles/) are single
# small-case launches whose algorithmic work is not known per launch, so the
# traffic field is null.
TRAFFIC = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="log2d_n65536")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--sparsify-prec", default="fp32", choices=["fp32", "fp64"],
                    help="precision of U, S, V on the mixed path (the FP64 path always sparsifies in FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--solver", default="gmres", choices=["gmres", "ir"],
                    help="outer iteration of the mixed path on the FP64 H^2 residual")
    return ap.parse_args()


def dist_setup(n):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"  # gloo: the host-side tests of this path
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(self.index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def kernel_source_hash(fname):
    src = open(os.path.join(ROOT, "paper_1705_04601_gb300", "csrc", fname), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


def roofline(prof, timed_launches_ok=True, sparsify_fp32=False):
    """Dominant kernel class by event time -> achieved vs its peak.

    The library's profiler records per class the algorithmic work of its
    launches: bytes for HBM-bound classes, flops for ALU-bound ones.
      gemm_update   tensor-core rank-64 update: HBM-bound, bytes (C read + written, L21, U12)
                    (H2SP_GEMM=simt: FP32 CUDA-core flops)
      panel, swap_trsm   FP32 flops (CUDA cores)
      transform, householder, coupling   FP64 flops (FP64 pipe), FP32 flops with an FP32 sparsification
      h2_matvec     FP64 flops (FP64 pipe)
      solve, apply, assemble, extend_add, vector    bytes
    """
    cls = max(prof, key=lambda c: prof[c]["ms"])
    p = prof[cls]
    per_launch_ms = p["ms"] / max(p["timed"], 1)
    work_per_launch = p["work"] / max(p["timed"], 1)
    peaks = measured_peaks()
    out = {"kernel": cls, "launches_timed": p["timed"], "avg_launch_ms": per_launch_ms}
    simt_gemm = os.environ.get("H2SP_GEMM", "") == "simt"
    sp_cls = ("transform", "householder", "coupling")
    if cls in ("panel", "swap_trsm") or (cls == "gemm_update" and simt_gemm) or (cls in sp_cls and sparsify_fp32):
        achieved = p["work"] / (p["ms"] * 1e-3) / 1e12
        out.update(bound="alu", achieved=achieved, peak=FP32_SIMT_TFLOPS, unit="TFLOP/s",
                   peak_source="derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (nominal max clock)")
    elif cls in sp_cls or cls == "h2_matvec":
        achieved = p["work"] / (p["ms"] * 1e-3) / 1e12
        out.update(bound="alu", achieved=achieved, peak=FP64_TFLOPS, unit="TFLOP/s",
                   peak_source="nominal GB300 FP64 (1.25 TFLOP/s); no measured FP64 peak available")
    else:
        achieved = p["work"] / (p["ms"] * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out.update(bound="hbm", achieved=achieved, peak=peak, unit="GB/s",
                   peak_source="measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback")
    out["frac"] = out["achieved"] / out["peak"]
    out["work_per_launch"] = work_per_launch
    tr = TRAFFIC.get(cls)
    valid = tr is not None and not simt_gemm and tr["src_hash"] == kernel_source_hash(tr["src"])
    out["traffic"] = tr["dram_over_algorithmic"] * work_per_launch if valid else None
    if valid:
        out["traffic_source"] = tr["capture"]
    return out


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1705_04601_gb300 import build
    from paper_1705_04601_gb300 import h2sp as H
    from paper_1705_04601_gb300 import synth

    build.build()
    t0 = time.time()
    h, b = synth.make_workload(args.workload)
    gen_s = time.time() - t0
    inp = H.H2Input(h)
    # symbolic analysis: once per structure, outside the timed steps
    ta = time.perf_counter()
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    analysis_ms = (time.perf_counter() - ta) * 1e3
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xt = torch.empty_like(bt)
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    mode = H.H2SP_GMRES if args.solver == "gmres" else H.H2SP_IR

    sp_flags = H.H2SP_SPARSIFY_FP32 if args.sparsify_prec == "fp32" else 0

    def mixed_step(profile=False):
        hd = H.h2sp_sparsify_analyzed(an, inp, flags=sp_flags)
        if profile:
            H.h2sp_profile(hd, timing=1, reset=True)
        H.h2sp_factor(hd, H.H2SP_FP32)
        info = H.h2sp_solve(hd, bt, xt, mode=mode, tol=1e-10, maxit=60, restart=20)
        return hd, info

    def fp64_step():
        # FP64 factorization; refinement on the FP64 H^2 residual stops as soon as 1e-10 holds
        hd = H.h2sp_sparsify_analyzed(an, inp)
        H.h2sp_factor(hd, H.H2SP_FP64)
        info64 = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=10)
        return hd, info64

    for _ in range(args.warmup):
        hd, info = mixed_step()
        hd.close()
    torch.cuda.synchronize()

    # ---- timed mixed steps (per-kernel events on the library's launch stream) ----
    clocks = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(ws)
    torch.cuda.synchronize()
    evs = [ev() for _ in range(args.steps + 1)]
    evs[0].record(stream)
    prof_sum, launches, infos, stats = None, 0, [], None
    # each step builds, factors and solves with its own handle; the handles
    # are read (per-kernel events) and released after the timed region, so
    # the host work of freeing them does not sit between two steps
    handles = []
    for k in range(args.steps):
        hd, info = mixed_step(profile=True)
        evs[k + 1].record(stream)
        handles.append(hd)
        infos.append((info.iters, info.rel_residual, info.status))
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    for hd in handles:
        pr = H.h2sp_profile(hd, timing=0)
        launches += sum(v["launches"] for v in pr.values())
        if prof_sum is None:
            prof_sum = {c: dict(v) for c, v in pr.items()}
            stats = H.h2sp_query(hd)
        else:
            for c, v in pr.items():
                for f in v:
                    prof_sum[c][f] += v[f]
        hd.close()
    del handles
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    mixed_s = max_over_ranks(sum(step_ms) / 1e3, ws) / args.steps
    x_mixed = xt.clone()

    # ---- FP64 direct path ----
    hd, _ = fp64_step()
    hd.close()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(args.fp64_steps):
        hd, info64 = fp64_step()
        if _ < args.fp64_steps - 1:
            hd.close()
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws) / args.fp64_steps
    # residual of the FP64 direct solution with the library's FP64 H^2 product
    yt = torch.empty_like(xt)
    H.h2sp_apply(hd, H.H2SP_OP_H2, xt, yt)
    res64 = float(((bt - yt).norm(dim=1) / bt.norm(dim=1)).max())
    diff = float((x_mixed - xt).norm() / xt.norm())
    hd.close()

    # ---- separate phase timing of one mixed step (outside the timed region) ----
    phase = {}
    e = [ev() for _ in range(4)]
    e[0].record(stream)
    hd = H.h2sp_sparsify_analyzed(an, inp, flags=sp_flags)
    e[1].record(stream)
    H.h2sp_factor(hd, H.H2SP_FP32)
    e[2].record(stream)
    H.h2sp_solve(hd, bt, xt, mode=mode, tol=1e-10, maxit=60, restart=20)
    e[3].record(stream)
    torch.cuda.synchronize()
    phase = {"sparsify_ms": e[0].elapsed_time(e[1]), "factor_fp32_ms": e[1].elapsed_time(e[2]),
             "refine_ms": e[2].elapsed_time(e[3]), "analysis_ms": analysis_ms}
    hd.close()
    # the FP64 factorization alone, for its GFLOP/s (also outside the timed region)
    e = [ev() for _ in range(3)]
    e[0].record(stream)
    hd = H.h2sp_sparsify_analyzed(an, inp)
    e[1].record(stream)
    H.h2sp_factor(hd, H.H2SP_FP64)
    e[2].record(stream)
    torch.cuda.synchronize()
    phase["sparsify_fp64_ms"] = e[0].elapsed_time(e[1])
    phase["factor_fp64_ms"] = e[1].elapsed_time(e[2])
    hd.close()

    # ---- e2e: host (pinned) buffers, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        names = ["leaf_basis", "transfer", "coupling", "near_block"]
        pinned = {nm: torch.from_numpy(np.ascontiguousarray(getattr(h, nm))).pin_memory() for nm in names}
        b_pin = torch.from_numpy(np.ascontiguousarray(b.T)).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        h2d = sum(t.numel() * 8 for t in pinned.values()) + b_pin.numel() * 8
        d2h = x_pin.numel() * 8

        def e2e_step():
            inp2 = H.H2Input(h, nonblocking_from=pinned)
            b2 = b_pin.cuda(non_blocking=True)
            x2 = torch.empty_like(b2)
            hd2 = H.h2sp_sparsify_analyzed(an, inp2, flags=sp_flags)
            H.h2sp_factor(hd2, H.H2SP_FP32)
            H.h2sp_solve(hd2, b2, x2, mode=mode, tol=1e-10, maxit=60, restart=20)
            x_pin.copy_(x2, non_blocking=True)
            return hd2, inp2

        hd2, _ = e2e_step()
        torch.cuda.synchronize()
        hd2.close()
        barrier(ws)
        a0, a1 = ev(), ev()
        a0.record(stream)
        keep = []
        for _ in range(args.steps):
            hd2, inp2 = e2e_step()
            keep.append((hd2, inp2))
        a1.record(stream)
        torch.cuda.synchronize()
        for hd2, _ in keep:
            hd2.close()
        e2e_s = max_over_ranks(a0.elapsed_time(a1) / 1e3, ws) / args.steps
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.workload)

    roof = roofline(prof_sum, sparsify_fp32=(args.sparsify_prec == "fp32"))
    fl = stats["factor_flops"]
    res_mixed = max(r for (_, r, _) in infos)
    out = {
        "metric": METRIC, "value": mixed_s, "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mixed_s * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": int(h.n), "leaf": 64, "basis_tol": 1e-6, "nrhs": int(b.shape[1]),
                   "kernel": "-log r", "points": "uniform [0,1]^2 (seeded)",
                   "l2": "inputs larger than L2 (443 MB of close blocks resident in HBM)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "sparsify_prec": args.sparsify_prec, "factor_prec": "fp32"},
        "mixed_s": mixed_s, "fp64_direct_s": fp64_s, "speedup_mixed_vs_fp64": fp64_s / mixed_s,
        "factor_flops": fl, "factor_gflops_fp32": None, "factor_gflops_fp64": None,
        "solver": args.solver, "refine_iters": [i for (i, _, _) in infos], "rel_residual_mixed": res_mixed, "rel_residual_fp64": res64,
        "fp64_refine_iters": info64.iters,
        "mixed_vs_fp64_rel_diff": diff, "phase_ms": phase, "input_gen_s": gen_s,
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches / max(args.steps, 1)),
        "kernel_ms_per_step": {c: v["ms"] / args.steps for c, v in prof_sum.items() if v["ms"] > 0},
        "clocks": clk, "cpu_baseline": cpu,
    }
    out["factor_gflops_fp32"] = fl / (phase["factor_fp32_ms"] * 1e-3) / 1e9
    out["factor_gflops_fp64"] = fl / (phase["factor_fp64_ms"] * 1e-3) / 1e9
    return out


def cpu_oracle_sample(workload, n=CPU_SAMPLE_N):
    """The oracle, as it stands, on the N=16384 instance of the same workload family."""
    import numpy as np

    from oracle import factor as ofa
    from oracle import sparsify as osp
    from paper_1705_04601_gb300 import synth
    h, b = synth.make_workload(workload, n=n)
    t0 = time.time()
    sp = osp.sparsify(h)
    fa = ofa.factor(h, sp)
    x = ofa.solve(h, sp, fa, b)
    dt = time.time() - t0
    assert np.all(np.isfinite(x))
    return {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle sparsify + FP64 block LU + direct solve (16 RHS) on the N=%d instance of the same "
                      "2D -log r workload (leaf<=64, basis tol 1e-6); not scaled to N=65536" % n}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import numpy as np

    from oracle import factor as ofa
    from oracle import sparsify as osp
    from paper_1705_04601_gb300 import synth
    h, b = synth.make_workload(args.workload, n=CPU_SAMPLE_N)

    def step():
        sp = osp.sparsify(h)
        fa = ofa.factor(h, sp)
        return ofa.solve(h, sp, fa, b)

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    for _ in range(args.steps):
        x = step()
    dt = (time.time() - t0) / args.steps
    assert np.all(np.isfinite(x))
    sample = ("oracle sparsify + FP64 block LU + direct solve (16 RHS) on the N=%d instance of the same 2D -log r "
              "workload (leaf<=64, basis tol 1e-6)" % CPU_SAMPLE_N)
    return {"impl": "reference", "metric": METRIC, "value": dt, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": CPU_SAMPLE_N, "sample_of_n": 65536},
            "cpu_baseline": {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": dt, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    ws, rank, local = dist_setup(args.gpus)
    out = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
