"""Autotuner of the launch shape: which cells go through the shared-memory
sort (and which through the multi-pass global path), which cells run one
warp per cell, and how many warps share a block.

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


def tune(runs, steps: int = 4, cache_path: str | None = DEFAULT_CACHE, candidates=None, force: bool = False) -> dict:
    """Times the candidates on `runs` (their state advances by the timed
    steps), sets the fastest process-wide and returns a report."""
    import torch

    cands = candidates or CANDIDATES
    key = f"{torch.cuda.get_device_name()}|{signature(runs)}"
    cache = _load(cache_path) if cache_path else {}
    if not force and key in cache:
        best = cache[key]["best"]
        sdm.sdm_set_tuning(best)
        return {"key": key, "best": best, "cached": True, "ms_per_step": cache[key].get("ms_per_step")}
    t0 = time.perf_counter()
    timings = []
    for c in cands:
        sdm.sdm_set_tuning(c)
        timings.append((time_candidate(runs, steps), c))
    timings.sort(key=lambda x: x[0])
    best_ms, best = timings[0]
    sdm.sdm_set_tuning(best)
    report = {"key": key, "best": best, "cached": False, "ms_per_step": best_ms,
              "worst_ms_per_step": timings[-1][0], "candidates": len(cands), "tuning_s": time.perf_counter() - t0}
    if cache_path:
        cache[key] = {"best": best, "ms_per_step": best_ms,
                      "all": [{"ms_per_step": t, **c} for t, c in timings]}
        _store(cache_path, cache)
    return report
