"""Autotuner of the FP32 block Cholesky's schedule.

The factorization's dense work is the block-end tensor-core update of every
front; how it shares the GPU with the panel stream depends on the front
sizes of the structure.  For one structure (an analysis handle) and one
device, ``tune`` times h2sp_factor(H2SP_FP32_CHOL) under candidate schedules
-- the h2sp_set_option knobs: the output tile of the block-end update (128 x
128, or 128 x 256 over pairs of column tiles), the most 128-column tiles one
CTA of it takes, the SMs that update leaves to the panel stream, and the
look-ahead -- by coordinate descent from the library's defaults, and
keeps the fastest.  A schedule changes the order of work, not the factors
beyond rounding order.

Choices persist as JSON, keyed by the device name and the structure's sizes
(points, supernodes, largest front, Cholesky flops): ``tuned.json`` beside
this file ships the choices made on a GB300, and ``$H2SP_TUNE_CACHE`` (if
set) names a file the tuner reads first and writes to.
"""
from __future__ import annotations

import json
import os

from . import h2sp as H

HERE = os.path.dirname(os.path.abspath(__file__))
SHIPPED = os.path.join(HERE, "tuned.json")
DEFAULT = {"tiles_per_cta": 0, "panel_sms": -1, "lookahead": 1, "wide": 2}
CANDIDATES = {
    "wide": [2, 1, 0],
    "tiles_per_cta": [0, 8, 16, 32, 64],
    "panel_sms": [-1, 8, 16, 32],
    "lookahead": [1, 0],
}
_OPT = {"tiles_per_cta": H.H2SP_OPTION_CHOL_TILES_PER_CTA, "panel_sms": H.H2SP_OPTION_CHOL_PANEL_SMS,
        "lookahead": H.H2SP_OPTION_CHOL_LOOKAHEAD, "wide": H.H2SP_OPTION_CHOL_WIDE}


def key(stats: dict, device: str) -> str:
    """Cache key: the device and the structure's sizes."""
    return "%s|n=%d|sn=%d|front=%d|chol=%.6e" % (device, stats["n"], stats["nsupernodes"], stats["max_front"],
                                                 stats["chol_flops"])


def _files():
    out = []
    env = os.environ.get("H2SP_TUNE_CACHE")
    if env:
        out.append(env)
    out.append(SHIPPED)
    return out


def load(k: str):
    """The stored schedule for key k, or None."""
    for f in _files():
        try:
            d = json.load(open(f))
        except (OSError, ValueError):
            continue
        if k in d:
            return dict(d[k]["schedule"])
    return None


def store(k: str, sched: dict, ms: float, path: str | None = None):
    path = path or os.environ.get("H2SP_TUNE_CACHE") or SHIPPED
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        d = {}
    d[k] = {"schedule": sched, "factor_ms": ms}
    with open(path, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)


def apply(hd: H.Handle, sched: dict | None):
    """Set a schedule on a handle (None: leave the defaults)."""
    if not sched:
        return
    for name, v in sched.items():
        H.h2sp_set_option(hd, _OPT[name], int(v))


def tune(an: H.Handle, inp: H.H2Input, flags: int = H.H2SP_SPARSIFY_FP32, repeats: int = 2, log=None):
    """Coordinate descent over CANDIDATES from DEFAULT; returns (schedule, ms).

    Each candidate factors a fresh numeric sparsification of the structure of
    ``an`` (the numbers of ``inp``) ``repeats`` times; its time is the best of
    those (CUDA events on the current stream)."""
    import torch

    hd = H.h2sp_sparsify_analyzed(an, inp, flags=flags)
    stream = torch.cuda.current_stream()

    def run(sched):
        apply(hd, sched)
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        if log:
            log("tune %s: %.2f ms" % (sched, best))
        return best

    H.h2sp_factor(hd, H.H2SP_FP32_CHOL)  # warm-up: buffers, descriptors
    try:
        return descend(run)
    finally:
        hd.close()


def descend(cost, default: dict | None = None, candidates: dict | None = None, margin: float = 0.99):
    """Coordinate descent: from ``default``, try each knob's candidate values
    in turn with the other knobs at the best schedule so far, and move only
    when the time ``cost(schedule)`` falls below ``margin`` times the best
    (run-to-run noise does not move it).  Returns (schedule, time)."""
    cur = dict(DEFAULT if default is None else default)
    cands = CANDIDATES if candidates is None else candidates
    cur_ms = cost(cur)
    for name, values in cands.items():
        for v in values:
            if v == cur[name]:
                continue
            cand = dict(cur, **{name: v})
            ms = cost(cand)
            if ms < cur_ms * margin:
                cur, cur_ms = cand, ms
    return cur, cur_ms
