#!/usr/bin/env python
"""Time to solution of A x = b at relative residual 1e-10 on one GB300.

One step = the whole hot path on one H^2 matrix with inputs resident in HBM:
the numeric sparsification h2sp_sparsify_analyzed (A = U S V^T), the
factorization of S (h2sp_factor) and the solve (h2sp_solve).  The host
analysis of the structure (h2sp_analyze: level schedule, block pattern of S,
symbolic factorization) runs once per structure, before the timed steps, and
is reported as ``analysis_ms``.

Default workload (the configuration the metric is stated on): 1/r on the
jittered Fibonacci sphere, N = 262,144, octree leaf <= 128, Chebyshev 4^3
bases recompressed to 1e-6, A_ii = 2 sqrt(N), one right-hand side.  S is
symmetric positive definite there, so S is factored by the block Cholesky
(--factor lu selects the block LU; the 2D -log r workloads need it).  Two
paths on the same inputs:

* mixed (the headline ``value``): S from FP32 sandwich products (the
  Householder completions stay FP64), FP32 factorization of S with FP32
  (three-term TF32) tensor-core updates, then restarted GMRES on the FP64 H^2
  product, right-preconditioned by V S^-1 U^T, until
  max_k ||b_k - A x_k|| / ||b_k|| <= 1e-10;
* fp64 (``fp64_direct_s``): FP64 sparsification and factorization, the
  direct solve refined on the FP64 H^2 residual to 1e-10.

``value`` comes from unprofiled steps; the per-kernel-class times and the
roofline come from one extra step with CUDA events around every launch.
``e2e`` repeats the mixed step through h2sp_solve_host from pinned host
buffers (all numeric H^2 arrays and b copied in, x copied out, inside the
timed region).  The close blocks (GBs) are larger than the 129 MB L2, so no
flush is needed between steps.

``--impl reference`` times the CPU FP64 oracle instead (the reference arm);
``cpu_baseline`` times it once.  Both run the oracle as it stands on the
N = 16,384 instance of the same workload (a bounded sample) and scale each
phase to the benched N by its algorithmic work (sparsification flops, factor
flops, factor entries for the solve).  Under torchrun every rank solves an
independent replica; rank 0 prints one JSON line.
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
DEFAULT_WORKLOAD = "inv3d_sphere_n262144"
CPU_SAMPLE_N = 16384
# workloads whose S is symmetric positive definite (1/r on the sphere with
# A_ii = 2 sqrt(N)): the block Cholesky applies
SPD_WORKLOADS = {"inv3d_sphere_n262144"}

# DRAM traffic of the dominant kernel from an ncu capture, per kernel class:
# dram bytes read + written of the captured launch divided by that launch's
# algorithmic work, valid while the kernel's source file is unchanged (sha256
# prefix of "src").  The bench's traffic figure is this ratio times the
# class's average work per launch.
TRAFFIC = {
    "gemm_update": {
        "src": "gemm_tc.cu", "src_hash": "b139c84ab103ed05", "dram_over_algorithmic": 0.016142,
        "capture": "profiles/gemm_tc_wide_inv3d_sphere_n32768.md: dram__bytes_read.sum + dram__bytes_write.sum over "
                   "every k_gemm_tc_wide launch (reduce-add epilogue, four stages) of two factorizations at N = 32,768 "
                   "(68.81 GB per factorization) divided by their algorithmic flops (4.263e12)",
    },
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="points (default: the workload's own N)")
    ap.add_argument("--factor", default="auto", choices=["auto", "chol", "lu"],
                    help="block Cholesky (SPD S) or block LU; auto: Cholesky on the SPD workloads")
    ap.add_argument("--fp64-steps", type=int, default=1, help="FP64 path steps timed (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--bf16-steps", type=int, default=2,
                    help="steps of the mixed path with BF16 block-end updates (reported beside the headline; 0: skip)")
    ap.add_argument("--sparsify-prec", default="fp32", choices=["fp32", "fp64"],
                    help="precision of the products into S on the mixed path (the FP64 path is FP64 throughout)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-construct", action="store_true",
                    help="skip the from-points variant (GPU H^2 construction + the mixed step)")
    ap.add_argument("--tune", default="auto", choices=["auto", "off", "force"],
                    help="schedule of the FP32 block Cholesky: auto = the stored choice for this device and "
                         "structure (paper_1705_04601_gb300/tuned.json), else tune now; off = library defaults")
    ap.add_argument("--solver", default="gmres", choices=["gmres", "ir"],
                    help="outer iteration of the mixed path on the FP64 H^2 residual")
    return ap.parse_args(argv)


def factor_kind(args):
    if args.factor != "auto":
        return args.factor
    return "chol" if args.workload in SPD_WORKLOADS else "lu"


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


def roofline(prof, fma_peaks, fp32_gemm_tc=True, sparsify_fp32=False):
    """Dominant kernel class by event time -> achieved vs its peak.

    The library's profiler records per class the algorithmic work of its
    launches (h2sp_kernel_times):
      gemm_update   the trailing update of the fronts, flops.  FP32 on the
                    tensor cores (three-term TF32 split, three MMAs per FP32
                    product): bound "tensor" against the three-pass ceiling
                    = measured BF16 dense rate x 0.5 (TF32 : BF16 nominal) / 3;
                    FP64 (or H2SP_GEMM=simt FP32): CUDA-core FMA pipe
      panel, swap_trsm   FP32 flops (CUDA cores)
      transform     FP64 flops (FP32 with an FP32 sparsification)
      h2_matvec     FP64 flops
      the others    bytes (HBM)
    fma_peaks: {"fp64": TFLOP/s, "fp32": TFLOP/s} measured by h2sp_measure_peak.
    """
    cls = max(prof, key=lambda c: prof[c]["ms"])
    p = prof[cls]
    per_launch_ms = p["ms"] / max(p["timed"], 1)
    work_per_launch = p["work"] / max(p["timed"], 1)
    peaks = measured_peaks()
    out = {"kernel": cls, "launches_timed": p["timed"], "avg_launch_ms": per_launch_ms}
    achieved_t = p["work"] / max(p["ms"] * 1e-3, 1e-30) / 1e12
    if cls == "gemm_update" and fp32_gemm_tc:
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        src = "measured (MEASURED_PEAKS.json bf16_tflops_sustained)" if bf16 else "fallback 1700 TFLOP/s bf16"
        bf16 = bf16 or 1700.0
        tf32 = 0.5 * bf16
        out.update(bound="tensor", achieved=achieved_t, peak=tf32 / 3.0, unit="TFLOP/s",
                   peak_source=src + " x 0.5 (TF32:BF16 nominal) / 3 (three TF32 MMAs per FP32 product)",
                   tf32_pipe_frac=3.0 * achieved_t / tf32)
    elif cls in ("gemm_update", "panel", "swap_trsm", "transform", "h2_matvec"):
        # the profiled step is the mixed one: its gemm_update here is the FP32 CUDA-core update
        fp64 = cls == "h2_matvec" or (cls == "transform" and not sparsify_fp32)
        key = "fp64" if fp64 else "fp32"
        out.update(bound="alu", achieved=achieved_t, peak=fma_peaks[key], unit="TFLOP/s",
                   peak_source="measured: h2sp_measure_peak %s FMA chains on every SM, CUDA events" % key.upper())
    else:
        achieved = p["work"] / max(p["ms"] * 1e-3, 1e-30) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out.update(bound="hbm", achieved=achieved, peak=peak, unit="GB/s",
                   peak_source="measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback")
    out["frac"] = out["achieved"] / out["peak"]
    out["work_per_launch"] = work_per_launch
    tr = TRAFFIC.get(cls)
    valid = tr is not None and tr["src_hash"] == kernel_source_hash(tr["src"])
    out["traffic"] = tr["dram_over_algorithmic"] * work_per_launch if valid else None
    if valid:
        out["traffic_source"] = tr["capture"]
    return out


def workload_config(name, n, nrhs, kind, sparsify_prec):
    from paper_1705_04601_gb300 import synth
    w = synth.WORKLOADS[name]
    kern = {"inv": "1/r", "log": "-log r", "yukawa": "exp(-r)/r"}[w["kernel"]]
    pts = {"sphere": "jittered Fibonacci sphere (seeded)"}.get(w.get("points", ""),
                                                                "uniform [0,1]^%d (seeded)" % w["dim"])
    return {"workload": name, "n": int(n), "leaf": w["leaf"], "basis_tol": w["tol"], "nrhs": int(nrhs),
            "kernel": kern, "points": pts, "factor": "block Cholesky" if kind == "chol" else "block LU",
            "sparsify_prec": sparsify_prec, "factor_prec": "fp32",
            "l2": "inputs larger than L2 (close blocks of several GB resident in HBM); no flush"}


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1705_04601_gb300 import build
    from paper_1705_04601_gb300 import h2sp as H
    from paper_1705_04601_gb300 import synth

    build.build()
    kind = factor_kind(args)
    prec32 = H.H2SP_FP32_CHOL if kind == "chol" else H.H2SP_FP32
    prec64 = H.H2SP_FP64_CHOL if kind == "chol" else H.H2SP_FP64
    t0 = time.time()
    h, b = synth.make_workload(args.workload, n=getattr(args, "n", None))
    gen_s = time.time() - t0
    inp = H.H2Input(h)
    # symbolic analysis: once per structure, outside the timed steps
    ta = time.perf_counter()
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    analysis_ms = (time.perf_counter() - ta) * 1e3
    stats = H.h2sp_query(an)
    fl32 = stats["chol_flops"] if kind == "chol" else stats["factor_flops"]
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xt = torch.empty_like(bt)
    stream = torch.cuda.current_stream()
    fma = {"fp64": H.h2sp_measure_peak(0), "fp32": H.h2sp_measure_peak(1)}
    sp_flags = H.H2SP_SPARSIFY_FP32 if args.sparsify_prec == "fp32" else 0
    # schedule of the FP32 block Cholesky: stored for this device and structure, or tuned now
    sched, sched_src, tune_s = None, "library defaults", 0.0
    if kind == "chol" and getattr(args, "tune", "auto") != "off":
        from paper_1705_04601_gb300 import tune as T
        tkey = T.key(dict(stats, n=int(h.n)), torch.cuda.get_device_name())
        sched = T.load(tkey) if args.tune == "auto" else None
        if sched is not None:
            sched_src = "stored (tuned.json)"
        else:
            t1 = time.time()
            sched, _ = T.tune(an, inp, flags=sp_flags)
            tune_s = time.time() - t1
            sched_src = "tuned in this run"
            if os.environ.get("H2SP_TUNE_STORE"):
                T.store(tkey, sched, _)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    mode = H.H2SP_GMRES if args.solver == "gmres" else H.H2SP_IR

    def mixed_step(profile=False, marks=None):
        if marks:
            marks[0].record(stream)
        hd = H.h2sp_sparsify_analyzed(an, inp, flags=sp_flags)
        if sched:
            from paper_1705_04601_gb300 import tune as T
            T.apply(hd, sched)
        if profile:
            H.h2sp_profile(hd, timing=1)
        if marks:
            marks[1].record(stream)
        H.h2sp_factor(hd, prec32)
        if marks:
            marks[2].record(stream)
        info = H.h2sp_solve(hd, bt, xt, mode=mode, tol=1e-10, maxit=60, restart=20)
        if marks:
            marks[3].record(stream)
        return hd, info

    for _ in range(args.warmup):
        hd, info = mixed_step()
        hd.close()
    torch.cuda.synchronize()

    # ---- timed mixed steps, unprofiled ----
    clocks = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(ws)
    torch.cuda.synchronize()
    evs = [ev() for _ in range(args.steps + 1)]
    evs[0].record(stream)
    infos = []
    launches = 0
    # each step builds, factors and solves with its own handle and releases it
    # (its fronts alone can be ~100 GB); the memory goes back to the
    # stream-ordered pool, which keeps it for the next step
    for k in range(args.steps):
        hd, info = mixed_step()
        evs[k + 1].record(stream)
        infos.append((int(info.iters), float(info.rel_residual), int(info.status)))
        launches += sum(v["launches"] for v in H.h2sp_profile(hd, timing=-1).values())
        hd.close()
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    mixed_s = max_over_ranks(sum(step_ms) / 1e3, ws) / args.steps
    res_mixed = max(r for (_, r, _) in infos)
    converged = all(st == H.H2SP_OK for (_, _, st) in infos) and res_mixed <= 1e-10
    x_mixed = xt.clone()

    # ---- the same mixed step with the block-end updates on BF16 tensor cores
    # (per-tile power-of-two scaling, FP32 accumulation; one BF16 term, or a
    # hi + lo split with three products): reported variants ----
    bf16_variants = {}
    bf16_kinds = [("mixed_bf16", "H2SP_BF16_CHOL", "one BF16 term"),
                  ("mixed_bf16x3", "H2SP_BF16X3_CHOL", "BF16 hi + lo split, three BF16 products")]
    for key, precname, what in bf16_kinds:
        if kind != "chol" or getattr(args, "bf16_steps", 2) <= 0:
            bf16_variants[key] = None
            continue
        try:
            def bf16_step(prec=getattr(H, precname)):
                hd = H.h2sp_sparsify_analyzed(an, inp, flags=sp_flags)
                if sched:
                    from paper_1705_04601_gb300 import tune as T
                    T.apply(hd, sched)
                H.h2sp_factor(hd, prec)
                info = H.h2sp_solve(hd, bt, xt, mode=mode, tol=1e-10, maxit=100, restart=30)
                info.compensated = int(H.h2sp_query(hd)["compensated_pivots"])
                hd.close()
                return info
            bf16_step()
            torch.cuda.synchronize()
            b0, b1 = ev(), ev()
            b0.record(stream)
            binfos = [bf16_step() for _ in range(args.bf16_steps)]
            b1.record(stream)
            torch.cuda.synchronize()
            ok = all(i.status == H.H2SP_OK and i.rel_residual <= 1e-10 for i in binfos)
            bf16_variants[key] = {
                "value": (b0.elapsed_time(b1) / 1e3 / args.bf16_steps) if ok else None, "unit": "s",
                "iters": [int(i.iters) for i in binfos], "rel_residual": max(float(i.rel_residual) for i in binfos),
                "compensated_pivots": max(i.compensated for i in binfos),
                "factor": "block Cholesky, block-end updates on BF16 tensor cores (%s) with a power-of-two scale "
                          "per 128-row tile of L21, FP32 accumulation" % what}
        except H.H2spError as e:
            bf16_variants[key] = {"value": None, "error": str(e)}

    # ---- one profiled mixed step: per-class event times, phases ----
    marks = [ev() for _ in range(4)]
    hd, _ = mixed_step(profile=True, marks=marks)
    torch.cuda.synchronize()
    prof = H.h2sp_profile(hd, timing=0)
    hd.close()
    phase = {"sparsify_ms": marks[0].elapsed_time(marks[1]), "factor_fp32_ms": marks[1].elapsed_time(marks[2]),
             "solve_ms": marks[2].elapsed_time(marks[3]), "analysis_ms": analysis_ms}

    # ---- FP64 path on the same inputs (phases timed inside the step) ----
    fp64_s, res64, info64, diff = None, None, None, None
    if args.fp64_steps > 0:
        tot = 0.0
        for _ in range(args.fp64_steps):
            m = [ev() for _ in range(4)]
            m[0].record(stream)
            hd = H.h2sp_sparsify_analyzed(an, inp)
            m[1].record(stream)
            H.h2sp_factor(hd, prec64)
            m[2].record(stream)
            info64 = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=10)
            m[3].record(stream)
            torch.cuda.synchronize()
            tot += m[0].elapsed_time(m[3]) / 1e3
            phase.update(sparsify_fp64_ms=m[0].elapsed_time(m[1]), factor_fp64_ms=m[1].elapsed_time(m[2]),
                         solve_fp64_ms=m[2].elapsed_time(m[3]))
            yt = torch.empty_like(xt)
            H.h2sp_apply(hd, H.H2SP_OP_H2, xt, yt)
            res64 = float(((bt - yt).norm(dim=1) / bt.norm(dim=1)).max())
            hd.close()
        fp64_s = max_over_ranks(tot, ws) / args.fp64_steps
        if info64.status != H.H2SP_OK or not (res64 <= 1e-10):
            fp64_s = None
        diff = float((x_mixed - xt).norm() / xt.norm())

    # ---- e2e: the whole path from pinned host buffers through h2sp_solve_host ----
    e2e = None
    if not args.no_e2e:
        names = ["leaf_basis", "transfer", "coupling", "near_block"]
        pinned = {nm: torch.from_numpy(np.ascontiguousarray(getattr(h, nm))).pin_memory() for nm in names}
        hinp = H.H2Input(h, device="host", host=pinned)
        b_pin = torch.from_numpy(np.ascontiguousarray(b.T)).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        h2d = sum(t.numel() * 8 for t in pinned.values()) + b_pin.numel() * 8
        d2h = x_pin.numel() * 8
        nr = int(b.shape[1])
        sh = torch.cuda.current_stream().cuda_stream

        def e2e_step():
            return H.h2sp_solve_host(an, hinp, b_pin.data_ptr(), h.n, x_pin.data_ptr(), h.n, nr, flags=sp_flags,
                                     prec=prec32, mode=mode, tol=1e-10, stream=sh)

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        ks = max(1, min(args.steps, args.e2e_steps))
        a0, a1 = ev(), ev()
        a0.record(stream)
        e2e_infos = [e2e_step() for _ in range(ks)]
        a1.record(stream)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(a0.elapsed_time(a1) / 1e3, ws) / ks
        ok = all(i.status == H.H2SP_OK and i.rel_residual <= 1e-10 for i in e2e_infos)
        e2e = {"value": e2e_s if ok else None, "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": ks, "entry": "h2sp_solve_host"}

    # ---- from points: the H^2 matrix built on the GPU (h2sp_construct, the
    # paper's "approx." step) from the same seeded points, then the mixed step
    # on it; the host tree and lists and the analysis of the built structure
    # stay outside the timed region ----
    from_points = None
    if not getattr(args, "no_construct", False):
        try:
            pts, plo, phi, pcfg = synth.workload_points(args.workload, n=int(h.n))
            t1 = time.time()
            tree, tp = synth.tree_arrays(pts, pcfg["leaf"], plo, phi)
            tree_s = time.time() - t1
            xp = torch.from_numpy(tp).cuda()
            diag = synth.default_diag(pcfg["kernel"], int(h.n), tp.shape[1])
            c0, c1 = ev(), ev()
            torch.cuda.synchronize()
            c0.record(stream)
            con = H.h2sp_construct(tree, xp, pcfg["kernel"], diag, order=4, tol=pcfg["tol"])
            c1.record(stream)
            torch.cuda.synchronize()
            construct_s = c0.elapsed_time(c1) / 1e3
            cd = con.desc()
            ncl = int(tree["parent"].size)
            crank = np.ctypeslib.as_array(cd.rank, shape=(ncl,)).copy()
            ta2 = time.perf_counter()
            an_c = H.h2sp_analyze(con)
            an_c_ms = (time.perf_counter() - ta2) * 1e3

            def points_step():
                hd = H.h2sp_sparsify_analyzed(an_c, con, flags=sp_flags)
                if sched:
                    from paper_1705_04601_gb300 import tune as T
                    T.apply(hd, sched)
                H.h2sp_factor(hd, prec32)
                info = H.h2sp_solve(hd, bt, xt, mode=mode, tol=1e-10, maxit=60, restart=20)
                hd.close()
                return info

            points_step()
            torch.cuda.synchronize()
            p0, p1 = ev(), ev()
            p0.record(stream)
            pinfo = points_step()
            p1.record(stream)
            torch.cuda.synchronize()
            step_s = p0.elapsed_time(p1) / 1e3
            ok = pinfo.status == H.H2SP_OK and pinfo.rel_residual <= 1e-10
            from_points = {
                "value": (construct_s + step_s) if ok else None, "unit": "s", "construct_s": construct_s,
                "step_s": step_s, "iters": int(pinfo.iters), "rel_residual": float(pinfo.rel_residual),
                "host_tree_s": tree_s, "analysis_ms": an_c_ms, "host_generator_s": gen_s,
                "ranks_equal_to_host_frac": float(np.mean(crank == np.asarray(h.rank))) if crank.size == h.rank.size
                else None,
                "what": "H^2 matrix built on the GPU (Chebyshev 4^d, recompressed to the workload's tolerance) "
                        "from the same points, then the mixed step on it",
            }
            an_c.close()
            con.close()
            del xp
        except H.H2spError as e:
            from_points = {"value": None, "error": str(e)}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(args.workload, kind, h)

    roof = roofline(prof, fma, fp32_gemm_tc=os.environ.get("H2SP_GEMM", "") != "simt",
                    sparsify_fp32=(args.sparsify_prec == "fp32"))
    out = {
        "metric": METRIC, "value": mixed_s if converged else None, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": dict(workload_config(args.workload, h.n, b.shape[1], kind, args.sparsify_prec),
                       parallelism="replicas" if ws > 1 else "single GPU"),
        "mixed_s": mixed_s, "converged": converged, "fp64_direct_s": fp64_s,
        "speedup_mixed_vs_fp64": (fp64_s / mixed_s) if (fp64_s and converged) else None,
        "factor_flops": fl32, "factor_gflops_fp32": fl32 / (phase["factor_fp32_ms"] * 1e-3) / 1e9,
        "factor_gflops_fp64": (fl32 / (phase["factor_fp64_ms"] * 1e-3) / 1e9) if "factor_fp64_ms" in phase else None,
        "solver": args.solver, "iters": [i for (i, _, _) in infos], "rel_residual_mixed": res_mixed,
        "rel_residual_fp64": res64, "fp64_refine_iters": info64.iters if info64 is not None else None,
        "mixed_vs_fp64_rel_diff": diff, "phase_ms": phase, "input_gen_s": gen_s,
        "structure": {"max_front": stats["max_front"], "nsupernodes": stats["nsupernodes"],
                      "nnz_S": stats["nnz"], "front_elems": stats["front_elems"]},
        "fma_peaks_tflops": fma, "roofline": roof, "e2e": e2e,
        "schedule": sched, "schedule_source": sched_src, "tune_s": tune_s, "mixed_bf16": bf16_variants["mixed_bf16"], "mixed_bf16x3": bf16_variants["mixed_bf16x3"],
        "gpu_launches": int(launches), "gpu_launches_per_step": int(launches / max(args.steps, 1)),
        "kernel_ms_per_step": {c: v["ms"] for c, v in prof.items() if v["ms"] > 0},
        "kernel_work_per_step": {c: v["work"] for c, v in prof.items() if v["ms"] > 0},
        "kernel_launches_per_step": {c: v["timed"] for c, v in prof.items() if v["ms"] > 0},
        "clocks": clk, "cpu_baseline": cpu, "from_points": from_points,
    }
    return out


def run_batched(args, ws, rank, local):
    """The batched form: many independent systems in one forest (one analysis,
    one handle).  A step is the persistent graph form: h2sp_refactor (graph
    replay of the numeric sparsification and the FP32 block LU of every
    system) + iterative refinement on the FP64 H^2 residual until every
    system's relative residual is <= 1e-10."""
    import numpy as np
    import torch

    from paper_1705_04601_gb300 import build
    from paper_1705_04601_gb300 import h2sp as H
    from paper_1705_04601_gb300 import synth

    build.build()
    w = synth.WORKLOADS[args.workload]
    nsys = getattr(args, "n", None) or w["n"]
    lo, hi = w["batched"]
    t0 = time.time()
    systems, forest, b = synth.make_batched(nsys, lo, hi, seed=synth.SEED_BASE + w["index"], leaf=w["leaf"],
                                            tol=w["tol"], nrhs=w["nrhs"])
    gen_s = time.time() - t0
    ta = time.perf_counter()
    an = H.h2sp_analyze(H.H2Input(forest, device=None))
    analysis_ms = (time.perf_counter() - ta) * 1e3
    stats = H.h2sp_query(an)
    inp = H.H2Input(forest)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xt = torch.empty_like(bt)
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # the persistent handle: built once, then every step replays its graph
    hd = H.h2sp_sparsify_analyzed(an, inp, flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32)

    def step():
        H.h2sp_refactor(hd)
        return H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    before = sum(v["launches"] for v in H.h2sp_profile(hd, timing=-1, reset=True).values())
    e0.record(stream)
    infos = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    launches = sum(v["launches"] for v in H.h2sp_profile(hd, timing=-1).values())
    del before
    t_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws) / args.steps
    res = max(float(i.rel_residual) for i in infos)
    converged = all(i.status == H.H2SP_OK for i in infos) and res <= 1e-10
    # phases of one step (outside the timed region)
    m = [ev() for _ in range(3)]
    m[0].record(stream)
    H.h2sp_refactor(hd)
    m[1].record(stream)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
    m[2].record(stream)
    torch.cuda.synchronize()
    phase = {"refactor_graph_ms": m[0].elapsed_time(m[1]), "refine_ms": m[1].elapsed_time(m[2]),
             "analysis_ms": analysis_ms, "refine_iters": int(info.iters)}
    # every system on its own: residual with its own H^2 product (the library's FP64 product on the forest)
    yt = torch.empty_like(xt)
    H.h2sp_apply(hd, H.H2SP_OP_H2, xt, yt)
    r = (bt - yt).cpu().numpy().T
    bb = b
    off = np.cumsum([0] + [s_.n for s_ in systems])
    per_sys = [float(np.linalg.norm(r[off[k]:off[k + 1]]) / np.linalg.norm(bb[off[k]:off[k + 1]]))
               for k in range(len(systems))]
    hd.close()
    # FP64 path: FP64 sparsification and block LU, refinement to 1e-10
    fp64_s = None
    if args.fp64_steps > 0:
        f0, f1 = ev(), ev()
        f0.record(stream)
        hd64 = H.h2sp_sparsify_analyzed(an, inp)
        H.h2sp_factor(hd64, H.H2SP_FP64)
        i64 = H.h2sp_solve(hd64, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=10)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_s = f0.elapsed_time(f1) / 1e3 if (i64.status == H.H2SP_OK and i64.rel_residual <= 1e-10) else None
        hd64.close()
    # e2e: the whole path from pinned host buffers
    e2e = None
    if not args.no_e2e:
        names = ["leaf_basis", "transfer", "coupling", "near_block"]
        pinned = {nm: torch.from_numpy(np.ascontiguousarray(getattr(forest, nm))).pin_memory() for nm in names}
        hinp = H.H2Input(forest, device="host", host=pinned)
        b_pin = torch.from_numpy(np.ascontiguousarray(b.T)).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        sh = torch.cuda.current_stream().cuda_stream

        def e2e_step():
            return H.h2sp_solve_host(an, hinp, b_pin.data_ptr(), forest.n, x_pin.data_ptr(), forest.n,
                                     int(b.shape[1]), flags=H.H2SP_SPARSIFY_FP32, prec=H.H2SP_FP32, mode=H.H2SP_IR,
                                     tol=1e-10, stream=sh)

        e2e_step()
        ks = max(1, min(args.steps, args.e2e_steps))
        a0, a1 = ev(), ev()
        a0.record(stream)
        oks = [e2e_step() for _ in range(ks)]
        a1.record(stream)
        torch.cuda.synchronize()
        ok = all(i.status == H.H2SP_OK and i.rel_residual <= 1e-10 for i in oks)
        e2e = {"value": (a0.elapsed_time(a1) / 1e3 / ks) if ok else None, "unit": "s",
               "h2d_bytes_per_step": int(sum(t.numel() * 8 for t in pinned.values()) + b_pin.numel() * 8),
               "d2h_bytes_per_step": int(x_pin.numel() * 8), "steps": ks, "entry": "h2sp_solve_host"}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_batched(systems, b)
    return {
        "metric": METRIC, "value": t_s if converged else None, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": int(forest.n), "nsys": len(systems), "n_k_range": [lo, hi],
                   "leaf": w["leaf"], "basis_tol": w["tol"], "kernel": "-log r", "points": "random ellipses (seeded)",
                   "factor": "block LU", "form": "persistent: h2sp_refactor graph replay + refinement",
                   "parallelism": "single GPU", "l2": "inputs larger than L2; no flush"},
        "converged": converged, "rel_residual_max": res, "rel_residual_per_system_max": max(per_sys),
        "iters": [int(i.iters) for i in infos], "fp64_direct_s": fp64_s,
        "speedup_mixed_vs_fp64": (fp64_s / t_s) if (fp64_s and converged) else None,
        "factor_flops": stats["factor_flops"], "phase_ms": phase, "input_gen_s": gen_s,
        "structure": {"max_front": stats["max_front"], "nsupernodes": stats["nsupernodes"],
                      "nfront_levels": stats["nfront_levels"]},
        "e2e": e2e, "gpu_launches": int(launches), "gpu_launches_per_step": int(launches / max(args.steps, 1)),
        "clocks": clk, "cpu_baseline": cpu, "roofline": None,
    }


def cpu_oracle_batched(systems, b, nsample=8):
    """The oracle on every (nsys / nsample)-th system, scaled to all systems
    by the oracle's own work counts (summed per phase)."""
    import numpy as np
    step = max(1, len(systems) // nsample)
    idx = list(range(0, len(systems), step))[:nsample]
    off = np.cumsum([0] + [s.n for s in systems])
    ph = [0.0, 0.0, 0.0]
    for k in idx:
        _, p = _oracle_step(systems[k], b[off[k]:off[k + 1]], "lu")
        ph = [a + c for a, c in zip(ph, p)]
    wall = [_oracle_work(s, "lu") for s in systems]
    ws_ = [wall[k] for k in idx]
    ratios = [sum(w[i] for w in wall) / max(sum(w[i] for w in ws_), 1e-300) for i in range(3)]
    return {"value": sum(t * r for t, r in zip(ph, ratios)), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle (FP64 sparsify + block LU + direct solve) on %d of the %d systems, phases %.2f / %.2f / "
                      "%.2f s, scaled to all systems by the oracle's work counts x %.1f / %.1f / %.1f"
                      % (len(idx), len(systems), ph[0], ph[1], ph[2], ratios[0], ratios[1], ratios[2])}


def _oracle_step(h, b, kind):
    """The oracle's pipeline, phase by phase: sparsify, factor, solve (FP64)."""
    from oracle import factor as ofa
    from oracle import sparsify as osp
    t0 = time.perf_counter()
    sp = osp.sparsify(h)
    t1 = time.perf_counter()
    fa = ofa.cholesky(h, sp) if kind == "chol" else ofa.factor(h, sp)
    t2 = time.perf_counter()
    if kind == "chol":
        c = osp.apply_T(sp, h, b, col=False)
        x = osp.apply_N(sp, h, ofa.solve_S_chol(fa, c), col=True)
    else:
        x = ofa.solve(h, sp, fa, b)
    t3 = time.perf_counter()
    return x, (t1 - t0, t2 - t1, t3 - t2)


def _oracle_work(h, kind):
    """Algorithmic work of the oracle's three phases on an H^2 matrix, from
    the oracle's own structure (no numerical work): the level schedule, the
    block pattern of S predicted from the close lists, and the symbolic
    factorization on it.  (sparsification: sum over each level's close pairs
    of m_t m_s (m_t + m_s); factor: flops of the block Cholesky / LU; solve:
    entries of the factors.)"""
    import types

    import numpy as np

    from oracle import factor as ofa
    from oracle import sparsify as osp
    sch = osp.schedule(h)
    sym = ofa.symbolic(h, types.SimpleNamespace(sch=sch, blocks=dict.fromkeys(osp.pattern_rule(h, sch))))
    m = sch.m
    wsp = 0.0
    for lev in range(sch.lstop):
        pr = sch.near[lev]
        if len(pr):
            mt, ms = m[pr[:, 0]].astype(float), m[pr[:, 1]].astype(float)
            wsp += float(np.sum(mt * ms * (mt + ms)))
    size = sch.node_size
    fl, ent = 0.0, 0.0
    for k in range(sym.sn_ptr.size - 1):
        sv = float(sum(size[int(v)] for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]))
        bv = float(sum(size[int(w)] for w in sym.boundary[k]))
        fl += (sv ** 3 / 3.0 + sv * sv * bv + sv * bv * bv) if kind == "chol" else \
            (2.0 / 3.0 * sv ** 3 + 2.0 * sv * sv * bv + 2.0 * sv * bv * bv)
        ent += sv * sv + 2.0 * sv * bv
    return wsp, fl, ent


def _work_ratios(h_full, h_sample, kind):
    wf, ws_ = _oracle_work(h_full, kind), _oracle_work(h_sample, kind)
    return tuple(a / b for a, b in zip(wf, ws_))


def cpu_oracle_sample(workload, kind, h_full, n=CPU_SAMPLE_N):
    """The oracle, as it stands, on the N = 16,384 instance of the same
    workload, each phase scaled to the benched N by its algorithmic work."""
    import numpy as np

    from paper_1705_04601_gb300 import synth
    hs, bs = synth.make_workload(workload, n=n)
    x, ph = _oracle_step(hs, bs, kind)
    assert np.all(np.isfinite(x))
    ratios = _work_ratios(h_full, hs, kind)
    nfull, nsamp = int(h_full.n), int(hs.n)
    scaled = sum(t * r for t, r in zip(ph, ratios))
    return {"value": scaled, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": ("oracle (FP64 sparsify + block %s + direct solve) on the N=%d instance of the same workload, "
                       "phases %.2f / %.2f / %.2f s, scaled to N=%d by algorithmic work x %.1f / %.1f / %.1f "
                       "(sparsification work, factor flops, factor entries, counted on the oracle's own schedule, block pattern "
                       "and symbolic factorization)"
                       % ("Cholesky" if kind == "chol" else "LU", nsamp, ph[0], ph[1], ph[2], nfull,
                          ratios[0], ratios[1], ratios[2])),
            "sample_phases_s": list(ph), "scale": list(ratios), "sample_n": nsamp}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import numpy as np

    from paper_1705_04601_gb300 import synth
    kind = factor_kind(args)
    w = synth.WORKLOADS[args.workload]
    if "batched" in w:
        # the sampled systems of the batched workload, each step scaled to all of them
        nsys = getattr(args, "n", None) or w["n"]
        lo_, hi_ = w["batched"]
        systems, forest, b = synth.make_batched(nsys, lo_, hi_, seed=synth.SEED_BASE + w["index"], leaf=w["leaf"],
                                                tol=w["tol"], nrhs=w["nrhs"])
        for _ in range(args.warmup):
            cpu_oracle_batched(systems, b)
        vals = [cpu_oracle_batched(systems, b) for _ in range(args.steps)]
        dt = sum(v["value"] for v in vals) / args.steps
        return {"impl": "reference", "metric": METRIC, "value": dt, "unit": "s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "n": int(forest.n), "nsys": len(systems)},
                "cpu_baseline": dict(vals[-1], value=dt),
                "e2e": {"value": dt, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    h, b = synth.make_workload(args.workload, n=CPU_SAMPLE_N)
    h_full, _ = synth.make_workload(args.workload, n=getattr(args, "n", None))  # its structure only enters the scaling
    ratios = _work_ratios(h_full, h, kind)
    nfull, nsamp = int(h_full.n), int(h.n)
    del h_full
    for _ in range(args.warmup):
        _oracle_step(h, b, kind)
    tot, ph_sum = 0.0, [0.0, 0.0, 0.0]
    for _ in range(args.steps):
        x, ph = _oracle_step(h, b, kind)
        tot += sum(t * r for t, r in zip(ph, ratios))
        ph_sum = [a + c for a, c in zip(ph_sum, ph)]
    dt = tot / args.steps
    assert np.all(np.isfinite(x))
    sample = ("oracle (FP64 sparsify + block %s + direct solve) on the N=%d instance of the same workload per step, "
              "phases scaled to N=%d by algorithmic work x %.1f / %.1f / %.1f"
              % ("Cholesky" if kind == "chol" else "LU", nsamp, nfull, ratios[0], ratios[1], ratios[2]))
    return {"impl": "reference", "metric": METRIC, "value": dt, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": nfull, "sample_n": nsamp,
                       "factor": "block Cholesky" if kind == "chol" else "block LU"},
            "cpu_baseline": {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample,
                             "sample_phases_s": [p / args.steps for p in ph_sum]},
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
    from paper_1705_04601_gb300 import synth
    if "batched" in synth.WORKLOADS.get(args.workload, {}):
        out = run_batched(args, ws, rank, local)
    else:
        out = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
