"""Autotuner of the launch shape: which cells go through the shared-memory
sort, which through the cluster path and which through the multi-pass global
path, which cells run one warp per cell, how many warps share a block, and
how many steps the warp-per-cell kernel fuses per launch.

The tuning never changes results: every candidate computes the same state bit
for bit.  The tuner times each candidate on the caller's own runs (one fused
batch, CUDA events, a few steps after a warm-up step) and keeps the fastest.
Results are cached in a JSON file keyed by the GPU name and a signature of
the workload (the histogram of stored cell sizes per kernel), so a second
batch of the same shape on the same GPU does not re-time.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import sdm

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sdm_gb300", "autotune.json")

CANDIDATES = [
    dict(smem_max_sd=s, warp_cell_max=w, warps_per_block=k)
    for s in (1024, 2048, 4096)
    for w in (0, 128, 256, 512)
    for k in ((2,) if w == 0 else (1, 2, 4))
]
MID_CHOICES = (0, 16384, 32768, 65536)  # largest cell on the cluster path (0: none)
FUSE_CHOICES = (0, 8, sdm.FUSE_STEPS_DEFAULT)
DEFAULT_SHAPE = dict(smem_max_sd=4096, warp_cell_max=512, warps_per_block=2)


def signature(runs) -> str:
    """Histogram of stored cell sizes (power-of-two classes) per kernel."""
    hist: dict[str, int] = {}
    for r in runs:
        info = r.info()
        # cells of a run share its layout; classes from the largest cell and count
        kind = "g" if r.cfg.kernel == 0 else "r"
        cls = int(np.ceil(np.log2(max(2, info.largest_cell))))
        key = f"{kind}{cls}"
        hist[key] = hist.get(key, 0) + int(info.n_cells)
    # bucket the counts so that similar workloads share an entry
    return ",".join(f"{k}:{int(2 ** np.round(np.log2(v)))}" for k, v in sorted(hist.items()))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_candidate(runs, steps: int) -> float:
    import torch

    batch = sdm.Batch(runs)
    batch.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(steps)
    e1.record()
    torch.cuda.synchronize()
    batch.close()
    return e0.elapsed_time(e1) / steps


def _search(runs, steps, cands, timings):
    out = []
    for c in cands:
        sdm.sdm_set_tuning(c)
        t = time_candidate(runs, steps)
        out.append((t, c))
        timings.append((t, c))
    return min(out, key=lambda x: x[0])


def tune(runs, steps: int = 4, cache_path: str | None = DEFAULT_CACHE, candidates=None, force: bool = False) -> dict:
    """Times candidates on `runs` (their state advances by the timed steps),
    sets the fastest process-wide and returns a report.  With `candidates`
    given, exactly those are timed; otherwise the search goes by stages: the
    cluster path's threshold with the default shape, then the shape (shared-
    memory threshold, warp classes, warps per block) with the best threshold,
    then the fused steps with the best of both."""
    import torch

    key = f"{torch.cuda.get_device_name()}|{signature(runs)}"
    cache = _load(cache_path) if cache_path else {}
    if not force and key in cache:
        best = cache[key]["best"]
        sdm.sdm_set_tuning(best)
        return {"key": key, "best": best, "cached": True, "ms_per_step": cache[key].get("ms_per_step")}
    t0 = time.perf_counter()
    timings = []
    if candidates:
        best_ms, best = _search(runs, steps, candidates, timings)
    else:
        fuse0 = sdm.FUSE_STEPS_DEFAULT
        _, b1 = _search(runs, steps, [dict(DEFAULT_SHAPE, mid_max_sd=m, fuse_steps=fuse0) for m in MID_CHOICES
                                      if m == 0 or m >= DEFAULT_SHAPE["smem_max_sd"]], timings)
        _, b2 = _search(runs, steps, [dict(c, mid_max_sd=b1["mid_max_sd"] if b1["mid_max_sd"] == 0 else
                                           max(b1["mid_max_sd"], c["smem_max_sd"]), fuse_steps=fuse0)
                                      for c in CANDIDATES], timings)
        best_ms, best = _search(runs, steps, [dict(b2, fuse_steps=f) for f in FUSE_CHOICES], timings)
    timings.sort(key=lambda x: x[0])
    sdm.sdm_set_tuning(best)
    report = {"key": key, "best": best, "cached": False, "ms_per_step": best_ms,
              "worst_ms_per_step": timings[-1][0], "candidates": len(timings), "tuning_s": time.perf_counter() - t0}
    if cache_path:
        cache[key] = {"best": best, "ms_per_step": best_ms,
                      "all": [{"ms_per_step": t, **c} for t, c in timings]}
        _store(cache_path, cache)
    return report
