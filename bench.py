"""Benchmark of the SDM coalescence step on the 4.19M-super-droplet grid.

Workload: 128 x 128 cells of dV = 1e3 m^3, 256 SDs per cell (4,194,304 SDs),
lognormal spectrum (geometric-mean radius 15 um, sigma_g 1.4, 1e8 m^-3),
geometric sweep-out kernel with Rogers-Yau fall speeds, dt = 1 s, FP64.  A
timed step is one coalescence step of every cell (one kernel launch); the
dv/dlnr product is taken once per 600 timed steps, as in the paper's usage
(run, then read the product), and its time is included.  The timed steps go
in turn to four independent runs of the grid (4 x 84 MB, more than twice the
L2), placed a quarter of a run apart, so that every 600 timed steps cover the
workload's own 600-step evolution once and a step's state was last touched
three steps (252 MB of other state) earlier.

value   pair-updates/s: sum over timed steps and cells of floor(n_c / 2),
        divided by the CUDA-event time of the sequences of steps (events
        around each sequence of up to 600 steps, not around each step) and
        of the spectra.
latency p50/p99 of one step, from a separate pass over one run with the L2
        flushed before every step (a 256 MiB write, then a 256 MiB read of
        another buffer) and an event pair around every step.
e2e     the same metric through the C ABI with host buffers: every step
        sdm_set_attributes from pinned host arrays, one step, and
        sdm_spectrum into host memory.
Multi-GPU (torchrun): every rank steps its own replica (weak scaling, no
collective on the data path).

``--impl reference`` times the oracle (plain C) on the host cores, one process
per core on 256 cells of the same workload each.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_17238_gb300 import inputs as I  # noqa: E402

METRIC = "SDM pair-updates/s & HBM roofline %; batched vs plain at equal accuracy; p50/p99"
UNIT = "pair-updates/s"
RUN_STEPS = 600
COPIES = 4  # state copies stepped in turn in the timed region (4 x 84 MB > 2 x L2)
WORKLOAD = ("grid_geometric: 128x128 cells x 256 SDs (4,194,304 SDs), dV=1e3 m^3, lognormal r_g=15um "
            "sigma_g=1.4 1e8 m^-3, geometric kernel (Rogers-Yau), dt=1 s, 600-step runs, FP64 p, int64 xi")
KERNEL_NAME = "warp_cell_step_kernel<256,2,2>"
PROFILE = os.path.join(ROOT, "profiles", "cell_step_kernel_grid_geometric_4M.md")
L2_FLUSH_BYTES = 256 << 20
EXTRAS = ("batched_vs_plain", "large_cells", "kfp32", "fused", "serving", "sedimentation", "long_kernel",
          "paper_setting", "condensation", "mid_cells")


# The step kernel and every helper it uses: the device header, and the kernel
# file up to the end of the warp-per-cell kernel (the large-cell path, the
# spectrum and the diagnostics follow it and do not change it).
KERNEL_SOURCES = (("sdm_device.cuh", None), ("sdm_kernels.cuh", b"// ----------------------------------------------------------- big cells"))


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_17238_gb300", "csrc")
    for f, end in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            text = fh.read()
        if end is not None:
            cut = text.find(end)
            if cut < 0:
                raise RuntimeError(f"{f}: end marker of the hashed region is missing")
            text = text[:cut]
        h.update(text)
    return h.hexdigest()[:16]


def profiled(key: str):
    """A per-launch figure (e.g. traffic_bytes_per_launch) from the committed
    ncu summary, if it was taken on the current kernel sources."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.eE+]+)", txt)
    hsh = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not hsh or hsh.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


def profiled_traffic():
    return profiled("traffic_bytes_per_launch")


SMS, SCHEDULERS_PER_SM = 152, 4


def issue_roofline(avg_kernel_s: float, sm_mhz):
    """The step kernel against the SMs' instruction issue rate: warp
    instructions per launch (ncu, the captured launch) over one instruction
    per scheduler per cycle on all SMs at the sampled SM clock."""
    inst = profiled("warp_instructions_per_launch")
    if inst is None or not sm_mhz:
        return None
    peak = SMS * SCHEDULERS_PER_SM * sm_mhz * 1e6  # warp instructions / s
    achieved = inst / avg_kernel_s
    return {"bound": "issue", "achieved": round(achieved / 1e9, 1), "peak": round(peak / 1e9, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions_per_launch": inst, "floor_us": round(inst / peak * 1e6, 2),
            "note": "instructions of the captured launch (the first timed step); later steps of a run issue more"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def max_over_ranks(t_local: float, dist=None, device=None) -> float:
    """The slowest rank's timed seconds (the whole job ends with it)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t_local
    import torch

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(pairs_per_replica_step: float, steps: int, world: int, t_max: float) -> float:
    """Pair-updates per second of all replicas together (weak scaling: every
    rank steps its own replica of the workload)."""
    return pairs_per_replica_step * steps * world / t_max


def replica_seed(rank: int) -> int:
    """Each rank's replica draws its own random streams."""
    return rank


def pairs_per_step(xi: np.ndarray, cell: np.ndarray, n_cells: int) -> int:
    live = np.bincount(cell[xi > 0], minlength=n_cells)
    return int((live // 2).sum())


# ------------------------------------------------------------------ our arm
def run_ours(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm

    B.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    g = I.grid_geometric(seed=replica_seed(rank))
    n_sd, n_cells = g.n_sd, g.n_cells
    cfg = lambda: sdm.make_config("geometric", "fp64", dv=g.dv, n_cells=n_cells, seed=g.seed)
    pairs0 = pairs_per_step(g.xi, g.cell, n_cells)
    xi_d = torch.from_numpy(g.xi).to(dev)
    v_d = torch.from_numpy(g.v).to(dev)
    cell_d = torch.from_numpy(g.cell).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2():
        flush.zero_()  # evicts every line of the state
        torch.sum(flush_r, dim=0, out=flush_sink)  # evicts the write's dirty lines (written back here)
    spec_d = torch.empty(len(I.R_EDGES) - 1, dtype=torch.float64, device=dev)

    def fresh_run(seed=None):
        r = sdm.Run(cfg() if seed is None else sdm.make_config("geometric", "fp64", dv=g.dv, n_cells=n_cells,
                                                                 seed=seed), n_sd)
        r.set_attributes(xi_d, v_d, cell_d)
        r.step(0)  # builds the launch plan (host work) before any timed event
        return r

    def positioned(c):
        # copy c: its own run (seed + c), advanced untimed to step c * RUN_STEPS / COPIES, so
        # that the copies' timed steps together cover one whole run
        r = fresh_run(g.seed + c)
        if c:
            r.step(c * (RUN_STEPS // COPIES))
        return r

    # warm-up (compiles nothing at run time; warms caches, allocator, clocks)
    run = fresh_run()
    for _ in range(args.warmup):
        run.step(1)
    run.spectrum(I.R_EDGES, out=spec_d)
    torch.cuda.synchronize()

    K = args.steps
    seq_ms = []
    spec_ms = []
    launches = 0
    sampler = ClockSampler(dev.index)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    done = 0
    runs = []
    # Inputs larger than L2: COPIES independent runs of the grid (4 x 84 MB), stepped in turn,
    # one launch per step; a step's state was last touched COPIES - 1 steps (252 MB of other
    # state) earlier.  Events bracket each sequence of steps, not each step.
    while done < K:
        for r in runs:
            r.close()
        runs = [positioned(c) for c in range(COPIES)]
        runs[-1].spectrum(I.R_EDGES, out=spec_d)  # its scratch allocated before the timed spectrum
        flush_l2()  # the untimed steps that placed the copies leave none of them in L2
        torch.cuda.synchronize()
        n = min(RUN_STEPS, K - done)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n):
            runs[i % COPIES].step(1)
        e1.record(stream)
        flush_l2()
        es = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es[0].record(stream)
        runs[-1].spectrum(I.R_EDGES, out=spec_d)
        es[1].record(stream)
        torch.cuda.synchronize()
        seq_ms.append(e0.elapsed_time(e1))
        spec_ms.append(es[0].elapsed_time(es[1]))
        launches += n + 2
        done += n
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    # pairs: live counts only fall when an SD dies; count them at the end of
    # the last copy (exact when equal to the start)
    xi_end, v_end = runs[-1].attributes()
    for r in runs:
        r.close()
    pairs_end = pairs_per_step(xi_end, g.cell, n_cells)
    pairs_avg = 0.5 * (pairs0 + pairs_end)
    total_ms = sum(seq_ms) + sum(spec_ms)
    t_local = total_ms / 1e3
    t_max = max_over_ranks(t_local, dist if world > 1 else None, dev)
    value = whole_job_value(pairs_avg, K, world, t_max)

    # per-step latency (untimed for the value): one run, L2 flushed before
    # every step outside the events, an event pair around every step
    step_ms = []
    run = fresh_run()
    torch.cuda.synchronize()
    nl = min(K, RUN_STEPS)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for i in range(nl):
        flush_l2()
        ev[i][0].record(stream)
        run.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]

    # writes per step (untimed replay of the same steps, counting changed SDs)
    written = count_written_bytes(run_factory=fresh_run, steps=min(K, RUN_STEPS), torch=torch, sdm=sdm,
                                  n_sd=n_sd)
    # algorithmic bytes of one step: the per-unit figure of the method's
    # statement (every live SD's multiplicity, volume and id read: 8 + 8 + 4 B,
    # the cells' offsets 8 B each, and the changed SDs' xi and v written) times
    # the units of one launch; this kernel reads no ids (an SD's random stream
    # is keyed by its rank in its cell), so it moves 16 B per SD, reported beside
    alg_bytes = 20 * n_sd + 8 * n_cells + written
    design_bytes = 16 * (n_sd + (n_sd % 2)) + 8 * n_cells + written
    avg_kernel_s = sum(seq_ms) / K / 1e3
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / avg_kernel_s / 1e9
    achieved_design = design_bytes / avg_kernel_s / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": profiled_traffic(),
                "kernel": KERNEL_NAME, "peak_kind": f"of {peak_kind}",
                "algorithmic_bytes_per_launch": int(alg_bytes),
                "algorithmic_bytes": "20 B per SD (xi, v, id) + 8 B per cell + the changed SDs' 16 B",
                "kernel_bytes_per_launch": int(design_bytes),
                "frac_of_kernel_bytes": round(achieved_design / peak, 4),
                "frac_of_nominal_8TBps": round(achieved / 8000.0, 4)}

    roofline["issue"] = issue_roofline(avg_kernel_s, clocks.get("sm_mhz") if isinstance(clocks, dict) else None)
    e2e = measure_e2e(args, g, sdm, torch, pairs0)
    run.close()
    extras = {}
    wanted = set() if args.no_extras else set(EXTRAS if args.extras == "all" else args.extras.split(","))
    if rank == 0:
        if "batched_vs_plain" in wanted:
            extras["batched_vs_plain"] = measure_batched_vs_plain(sdm, torch)
        if "large_cells" in wanted:
            extras["large_cells"] = measure_large_cells(sdm, torch)
        if "kfp32" in wanted:
            extras["kfp32"] = measure_kfp32(sdm, torch, g)
        if "fused" in wanted:
            extras["fused"] = measure_fused(sdm, torch, g)
        if "serving" in wanted:
            extras["serving"] = measure_serving(torch, args.serve_requests)
        if "sedimentation" in wanted:
            extras["sedimentation"] = measure_sedimentation(sdm, torch, g)
        if "long_kernel" in wanted:
            extras["long_kernel"] = measure_long_kernel(sdm, torch, g)
        if "paper_setting" in wanted:
            extras["paper_setting"] = measure_paper_setting(sdm, torch)
        if "condensation" in wanted:
            extras["condensation"] = measure_condensation(sdm, torch, g)
        if "mid_cells" in wanted:
            extras["mid_cells"] = measure_mid_cells(sdm, torch)
    res = None
    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded lognormal constant-multiplicity sample)",
            "config": {"workload": WORKLOAD, "n_sd": n_sd, "n_cells": n_cells, "pairs_per_step": pairs0,
                       "l2": f"inputs larger than L2: {COPIES} independent runs of the grid ({COPIES} x 84 MB) "
                             "stepped in turn, one launch per step, so a step's state was last touched "
                             f"{COPIES - 1} steps ({(COPIES - 1) * 84} MB of other state) before; CUDA events around "
                             "each sequence of steps; the spectrum after an L2 flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency_ms": {"p50": percentile(step_ms, 50), "p99": percentile(step_ms, 99),
                           "mean": statistics.mean(step_ms), "spectrum_ms": statistics.mean(spec_ms),
                           "note": "one run, L2 flushed before every step outside the events, an event pair "
                                   "around every step (an event pair adds about 2 us to a step)"},
            "roofline": roofline,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": launches,
            "wall_s_timed_region": wall,
        }
        res.update(extras)
    return res


def count_written_bytes(run_factory, steps, torch, sdm, n_sd):
    run = run_factory()
    dev = torch.device("cuda", torch.cuda.current_device())
    xi_prev = torch.empty(n_sd, dtype=torch.int64, device=dev)
    v_prev = torch.empty(n_sd, dtype=torch.float64, device=dev)
    xi_cur = torch.empty_like(xi_prev)
    v_cur = torch.empty_like(v_prev)
    sdm.sdm_get_attributes(run.h, xi=xi_prev, volume=v_prev)
    total = 0
    for _ in range(steps):
        run.step(1)
        sdm.sdm_get_attributes(run.h, xi=xi_cur, volume=v_cur)
        total += 8 * int((xi_cur != xi_prev).sum().item()) + 8 * int((v_cur != v_prev).sum().item())
        xi_prev, xi_cur = xi_cur, xi_prev
        v_prev, v_cur = v_cur, v_prev
    run.close()
    return total / steps


def measure_e2e(args, g, sdm, torch, pairs0):
    """set_attributes from pinned host buffers + one step + spectrum to host."""
    n = max(3, min(args.steps, 50))
    xi_h = torch.from_numpy(g.xi).pin_memory()
    v_h = torch.from_numpy(g.v).pin_memory()
    c_h = torch.from_numpy(g.cell).pin_memory()
    out = torch.empty(len(I.R_EDGES) - 1, dtype=torch.float64).pin_memory()
    run = sdm.Run(sdm.make_config("geometric", "fp64", dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
    for _ in range(2):
        run.set_attributes(xi_h, v_h, c_h).step(1)
        run.spectrum(I.R_EDGES, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        run.set_attributes(xi_h, v_h, c_h)
        run.step(1)
        run.spectrum(I.R_EDGES, out=out)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / n
    # a whole run through the same calls: one upload, the 600 steps in one
    # call (default launch tuning), the spectrum back; host wall time
    steps = g.steps or 600
    pairs_run = pairs_per_step(g.xi, g.cell, g.n_cells) * steps  # pairs of the initial state, every step
    t0 = time.perf_counter()
    run.set_attributes(xi_h, v_h, c_h)
    run.step(steps)
    run.spectrum(I.R_EDGES, out=out)
    torch.cuda.synchronize()
    dt_run = time.perf_counter() - t0
    run.close()
    h2d = g.n_sd * (8 + 8 + 4)
    # the host link itself: one plain pinned copy of the same bytes, for scale
    dev = torch.device("cuda", torch.cuda.current_device())
    src = torch.empty(h2d, dtype=torch.uint8).pin_memory()
    dst = torch.empty(h2d, dtype=torch.uint8, device=dev)
    dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        dst.copy_(src, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    link_gbs = 5 * h2d / (e0.elapsed_time(e1) * 1e-3) / 1e9
    return {"value": pairs0 / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "pinned_h2d_copy_gbs": link_gbs,
            "d2h_bytes_per_step": 8 * (len(I.R_EDGES) - 1), "ms_per_step": dt * 1e3, "steps": n,
            "whole_run": {"steps": steps, "ms": dt_run * 1e3, "ms_per_step": dt_run * 1e3 / steps,
                          "pair_updates_per_s": pairs_run / dt_run,
                          "note": "one set_attributes from pinned host memory, one call of all steps, "
                                  "the spectrum to host; host wall time"}}


def _timed(torch, fn):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def measure_batched_vs_plain(sdm, torch, steps=20):
    """1024 Golovin boxes, n_sd = round(2^U(8,16)): one fused batch (CUDA graph)
    against one context stepped after another.  The batch runs once with the
    default launch tuning and once with the autotuner's pick (timed on a
    separate copy of the ensemble).  FP64 states of all forms are identical
    bit for bit (checked), so accuracy is equal by construction.  State (~12M
    SDs, ~190 MB) exceeds L2; no flush needed."""
    from paper_2103_17238_gb300 import autotune

    insts = I.batched_ensemble(steps=steps)
    pairs = sum(pairs_per_step(t.xi, t.cell, t.n_cells) for t in insts)
    mk = lambda t: sdm.Run(sdm.make_config("golovin", dv=t.dv, seed=t.seed), t.n_sd).set_attributes(
        t.xi, t.v, t.cell)
    probe = [mk(t) for t in insts]
    rep = autotune.tune(probe, steps=3, cache_path=None)
    for r in probe:
        r.close()
    best = rep["best"]

    runs_b = [mk(t) for t in insts]
    runs_p = [mk(t) for t in insts]
    times = {}
    for name, tuning in (("default", None), ("tuned", best)):
        sdm.sdm_set_tuning(tuning)
        batch = sdm.Batch(runs_b, use_graph=True, graph_steps=10)
        batch.step(10)  # warm-up (captures the graph)
        times[name] = _timed(torch, lambda: batch.step(steps))
        batch.close()
    # plain contexts build their plans at their first step: with the pick
    for r in runs_p:
        r.step(10)

    def plain():
        for _ in range(steps):
            for r in runs_p:
                r.step(1)

    tp = _timed(torch, plain)
    for r in runs_p:
        r.step(10 + steps)
    sdm.sdm_set_tuning(None)
    same = all(np.array_equal(a.attributes()[0], b.attributes()[0]) and
               np.array_equal(a.attributes()[1], b.attributes()[1]) for a, b in zip(runs_b[:64], runs_p[:64]))
    for r in runs_b + runs_p:
        r.close()
    tb = times["tuned"]
    return {"workload": "1024 Golovin boxes, n_sd=round(2^U(8,16)) (rng 3), seeds 0..1023, FP64",
            "sd_total": int(sum(t.n_sd for t in insts)), "steps": steps,
            "batched_pair_updates_per_s": pairs * steps / tb,
            "batched_default_tuning_pair_updates_per_s": pairs * steps / times["default"],
            "plain_pair_updates_per_s": pairs * steps / tp,
            "speedup": tp / tb, "autotune": {"best": best, "candidates": rep["candidates"],
                                             "tuning_s": round(rep["tuning_s"], 2)},
            "equal_accuracy": "bit-identical states" if same else "MISMATCH"}


def measure_large_cells(sdm, torch, steps=10, members=32):
    """32 ensemble members of the 2^20-SD single-cell Golovin box, batched."""
    runs = []
    pairs = 0
    for seed in range(members):
        t = I.box_golovin(2**20, seed=seed)
        pairs += pairs_per_step(t.xi, t.cell, t.n_cells)
        runs.append(sdm.Run(sdm.make_config("golovin", dv=t.dv, seed=seed), t.n_sd).set_attributes(t.xi, t.v, t.cell))
    batch = sdm.Batch(runs)
    batch.step(2)
    dt = _timed(torch, lambda: batch.step(steps))
    batch.close()
    for r in runs:
        r.close()
    return {"workload": "32 x Golovin box n_sd=2^20 (one cell each), FP64; state 540 MB > L2",
            "pair_updates_per_s": pairs * steps / dt, "ms_per_step": dt / steps * 1e3}


def measure_sedimentation(sdm, torch, g, steps=50):
    """The grid as 128 columns x 128 levels of 10 m, dt = 1 s: a
    sedimentation step (fall, regroup, new layout) then a coalescence step.
    Device times by CUDA events; the coupled step's wall time includes the
    host's read of the new cell offsets and the launch plan it rebuilds.
    Algorithmic bytes of the sedimentation step: the whole layout read and
    written once (xi, v, zeta, id: 28 B per SD each way)."""
    nx, dz = 128, 10.0
    rng = np.random.default_rng(12)
    z = (g.cell // nx).astype(np.float64) * dz + rng.uniform(0.0, dz, g.n_sd)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell).set_positions(z, nx, dz)
    _, cell0 = run.positions(want_z=False)
    for _ in range(3):
        run.sediment()
        run.step(1)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    precip = 0.0
    t0 = time.perf_counter()
    for e in ev:
        e[0].record()
        precip += run.sediment()
        e[1].record()
        e[2].record()
        run.step(1)
        e[3].record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / steps
    sed_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    coal_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in ev)
    _, cell1 = run.positions(want_z=False)
    moved = float(np.mean(cell1 != cell0))
    run.close()
    gbs = 56.0 * g.n_sd / (sed_ms * 1e-3) / 1e9
    return {"workload": "grid_geometric 4,194,304 SDs as 128 columns x 128 levels of 10 m, dt = 1 s, heights "
                        "uniform in each level (rng 12); sedimentation then coalescence per step",
            "steps": steps, "sedimentation_ms": sed_ms, "coalescence_ms": coal_ms,
            "coupled_wall_ms": wall * 1e3, "sedimentation_algorithmic_gbs": gbs,
            "sedimentation_frac_of_measured_hbm": gbs / measured_peaks()[0],
            "sds_changed_cell_over_run": moved, "precipitated_m3": precip}


def measure_kfp32(sdm, torch, g, steps=600):
    """The grid with K and p in binary32: throughput, and the dv/dlnr spectrum
    after 600 steps against the binary64 run (which matches the oracle bit
    for bit)."""
    out = {}
    specs = {}
    for prec in ("fp64", "kfp32"):
        run = sdm.Run(sdm.make_config("geometric", prec, dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
        run.set_attributes(g.xi, g.v, g.cell).step(0)
        dt = _timed(torch, lambda: run.step(steps))
        specs[prec] = run.spectrum(I.R_EDGES)
        out[prec + "_pair_updates_per_s"] = pairs_per_step(g.xi, g.cell, g.n_cells) * steps / dt
        run.close()
    a, b = specs["fp64"], specs["kfp32"]
    out["spectrum_rel_l1_kfp32_vs_fp64"] = float(np.abs(b - a).sum() / np.abs(a).sum())
    out["steps"] = steps
    out["note"] = ("one 600-step call per precision under the default launch tuning (fused launches of "
                   f"{sdm.FUSE_STEPS_DEFAULT} steps); state resident, no L2 flush between steps (state 67 MB)")
    return out


def measure_fused(sdm, torch, g, steps=600):
    """The grid's whole 600-step run in one call: one launch per step against
    fused launches that keep every cell in shared memory for 8, 32 or 600
    steps.  The final states must be identical."""
    pairs = pairs_per_step(g.xi, g.cell, g.n_cells)
    out = {"steps": steps, "note": "one sdm_coalescence_step call of 600 steps; state resident, no L2 flush"}
    ref = None
    try:
        for f in (0, 8, 32, 600):
            sdm.sdm_set_tuning({"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": f})
            run = sdm.Run(sdm.make_config("geometric", "fp64", dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
            run.set_attributes(g.xi, g.v, g.cell).step(0)
            dt = _timed(torch, lambda: run.step(steps))
            xi, v = run.attributes()
            run.close()
            key = "per_step_launch" if f == 0 else f"fuse_{f}"
            out[key + "_pair_updates_per_s"] = pairs * steps / dt
            out[key + "_ms_per_step"] = dt * 1e3 / steps
            if ref is None:
                ref = (xi, v)
            else:
                out[key + "_state_identical"] = bool(np.array_equal(xi, ref[0]) and np.array_equal(v, ref[1]))
    finally:
        sdm.sdm_set_tuning(None)
    return out


def measure_mid_cells(sdm, torch, steps=10):
    """Mid-size cells, one cluster size at a time, filling the GPU once: 152
    Golovin boxes of 12,000 SDs (one CTA each), 72 of 24,000 (clusters of
    2), 36 of 60,000 (clusters of 4; 36 such clusters fit at once), each
    through the cluster path and through the multi-pass global path
    (tuning mid_max_sd 65536 and 0, one launch per step).  The states of the
    two paths are compared bit for bit."""
    out = {"workload": "Golovin boxes (b=1500 s^-1, dV=1e6 m^3), one cell each, seeds 0.., one launch per step",
           "steps": steps}
    base = {"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": 0}
    try:
        for n_sd, cells, k in ((12000, 152, 1), (24000, 72, 2), (60000, 36, 4)):
            res, states = {}, []
            for name, mid in (("cluster", 65536), ("multi_pass", 0)):
                sdm.sdm_set_tuning({**base, "mid_max_sd": mid})
                runs = [sdm.Run(sdm.make_config("golovin", dv=I.DV_BOX, seed=c), n_sd).set_attributes(
                    *(lambda t: (t.xi, t.v, t.cell))(I.box_golovin(n_sd, seed=c))) for c in range(cells)]
                batch = sdm.Batch(runs)
                batch.step(2)
                dt = _timed(torch, lambda: batch.step(steps))
                batch.close()
                states.append([r.attributes() for r in runs[:8]])
                for r in runs:
                    r.close()
                res[name + "_us_per_step"] = dt / steps * 1e6
                res[name + "_pair_updates_per_s"] = cells * (n_sd // 2) * steps / dt
            res["identical"] = all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
                                   for a, b in zip(*states))
            out[f"K{k}_{cells}x{n_sd}"] = res
    finally:
        sdm.sdm_set_tuning(None)
    return out


def measure_long_kernel(sdm, torch, g, steps=200):
    """The grid with Long's (1974) collision efficiency on the geometric
    kernel: one launch per step with L2 flushed between steps (as the
    headline), FP64 and KFP32."""
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)
    pairs = pairs_per_step(g.xi, g.cell, g.n_cells)
    out = {"workload": "grid_geometric 4,194,304 SDs, geometric sweep-out x Long (1974) efficiency, first "
                       f"{steps} steps, one launch per step, L2 flushed between steps", "steps": steps}
    for prec in ("fp64", "kfp32"):
        run = sdm.Run(sdm.make_config("long", prec, dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
        run.set_attributes(g.xi, g.v, g.cell).step(0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            torch.sum(flush_r, dim=0, out=sink)
            a.record()
            run.step(1)
            b.record()
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        xi, _ = run.attributes()
        run.close()
        out[prec] = {"pair_updates_per_s": pairs / (ms * 1e-3), "ms_per_step": ms,
                     "sds_changed": int((xi != g.xi).sum())}
    return out


def measure_condensation(sdm, torch, g, steps=100):
    """The condensation step on the grid (4.19M SDs, a supersaturation field
    of +-2% over the cells), one call per step with L2 flushed between
    steps, without and with the per-cell condensed-water output.
    Algorithmic bytes: xi and v read (16 B) and v written (8 B) per SD."""
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)
    rng = np.random.default_rng(5)
    G = np.full(g.n_cells, 1.1e-10)
    s = rng.uniform(-0.02, 0.02, g.n_cells)
    out_d = torch.empty(g.n_cells, dtype=torch.float64, device=dev)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell)
    peak = measured_peaks()[0]
    out = {"workload": "grid_geometric 4,194,304 SDs, G = 1.1e-10 m^2/s, s uniform in [-0.02, 0.02] per cell "
                       "(rng 5), dt = 1 s, r_min = 1 um; one call per step, L2 flushed between steps",
           "steps": steps, "algorithmic_bytes_per_sd": 24}
    for name, want in (("update_only", False), ("with_condensed", True)):
        for _ in range(3):
            sdm.sdm_condensation_step(run.h, G, s, 1e-6, out=out_d if want else None, want_condensed=False,
                                      n_cells=g.n_cells)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            torch.sum(flush_r, dim=0, out=sink)
            a.record()
            sdm.sdm_condensation_step(run.h, G, s, 1e-6, out=out_d if want else None, want_condensed=False,
                                      n_cells=g.n_cells)
            b.record()
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        gbs = 24.0 * g.n_sd / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_step": ms, "algorithmic_gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                     "sd_updates_per_s": g.n_sd / (ms * 1e-3)}
    run.close()
    return out


def measure_paper_setting(sdm, torch, seeds=8):
    """The paper's Golovin box (API in brief, Fig. 1): n_sd = 2^17 (and 2^12
    for comparison), dt = 1 s, 3600 steps, 8 seeds in one batch; relative L1
    error of the ensemble-mean dv/dlnr against the closed form's bin averages
    (bins holding >= 1e-3 of the peak) and N(t) / N_closed_form - 1 at
    t = 1200, 2400, 3600 s.  Time: the batch's 3600 steps (CUDA events)."""
    from oracle import golovin as G

    t_out = [1200, 2400, 3600]
    x0 = I.x0_box()
    out = {"workload": "Golovin box b=1500 s^-1, dV=1e6 m^3, dt=1 s, 3600 steps, 8 seeds batched", "seeds": seeds}
    for n_sd in (2**12, 2**17):
        g = I.box_golovin(n_sd)
        runs = [sdm.Run(sdm.make_config("golovin", "fp64", dv=I.DV_BOX, seed=s), n_sd).set_attributes(g.xi, g.v, g.cell)
                for s in range(seeds)]
        batch = sdm.Batch(runs, use_graph=True, graph_steps=100)
        done, step_s = 0, 0.0
        res = {}
        live = [seeds * n_sd]  # live SDs at 0 and at each output time
        for t in t_out:
            step_s += _timed(torch, lambda: batch.step(t - done))
            done = t
            spec = np.mean([r.spectrum(I.R_EDGES) for r in runs], axis=0)
            diags = [r.diagnostics() for r in runs]
            live.append(sum(d["live_sd"] for d in diags))
            num = np.mean([d["sum_xi"] / I.DV_BOX for d in diags])
            want = G.dv_dlnr_bins(I.R_EDGES, t, b=I.GOLOVIN_B, n0=I.N_CONC_BOX, x0=x0)
            mask = want >= 1e-3 * want.max()
            res[f"t{t}"] = {"spectrum_rel_l1": float(np.abs(spec[mask] - want[mask]).sum() / want[mask].sum()),
                            "number_rel_err": float(num / G.total_number(t, b=I.GOLOVIN_B, n0=I.N_CONC_BOX,
                                                                         x0=x0) - 1.0)}
        batch.close()
        for r in runs:
            r.close()
        res["ms_per_step"] = step_s / 3600 * 1e3
        # pairs per step from the live counts at the output times (trapezoid)
        pairs = sum(0.5 * (a + b) / 2 * (t1 - t0) for a, b, t0, t1 in zip(live[:-1], live[1:], [0] + t_out[:-1], t_out))
        res["pair_updates_per_s"] = pairs / step_s
        out[f"n_sd_2^{int(round(math.log2(n_sd)))}"] = res
    return out


def measure_serving(torch, n_requests=200):
    from paper_2103_17238_gb300 import serve

    reqs = I.serving_stream(n_requests=n_requests)
    srv = serve.Server(budget_bytes=120 * 10**9, chunk=20, fuse_steps=0)  # one launch per step
    res = srv.serve(reqs)
    out = {"workload": f"{n_requests} Poisson arrivals at 200/s (rng 4): Golovin boxes or geometric grids, "
                       "n_sd=round(2^U(10,20)), 100-1000 steps, dt in {0.5,1,2}; HBM budget 120 GB; "
                       "ticks of up to 20 steps, one launch per step",
           "pair_updates_per_s": res["pair_updates_per_s"], "step_latency_ms": res["step_latency_ms"],
           "time_in_system_s": res["time_in_system_s"], "requests": res["requests"],
           "max_active": res["max_active"], "wall_s": res["wall_s"]}
    # the same stream with each tick's steps fused for the cells of up to 512 SDs
    res = serve.Server(budget_bytes=120 * 10**9, chunk=20, fuse_steps=20).serve(reqs)
    out["fused_ticks"] = {"pair_updates_per_s": res["pair_updates_per_s"], "step_latency_ms": res["step_latency_ms"],
                          "time_in_system_s": res["time_in_system_s"], "max_active": res["max_active"]}
    # capacity: the same requests arriving all at once (arrival times / 1e6),
    # so that the device, not the arrival process, sets the rate
    for name, fuse in (("saturated", 0), ("saturated_fused_ticks", 20)):
        res = serve.Server(budget_bytes=120 * 10**9, chunk=20, fuse_steps=fuse, time_scale=1e6).serve(reqs)
        out[name] = {"requests_per_s": res["requests_per_s"], "pair_updates_per_s": res["pair_updates_per_s"],
                     "pair_updates_per_device_s": res["pair_updates_per_device_s"],
                     "step_latency_ms": res["step_latency_ms"], "time_in_system_s": res["time_in_system_s"],
                     "max_active": res["max_active"], "wall_s": res["wall_s"], "device_busy_s": res["device_busy_s"]}
    return out


def percentile(xs, q):
    s = sorted(xs)
    if not s:
        return None
    k = (len(s) - 1) * q / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return s[lo] + (s[hi] - s[lo]) * (k - lo)


CPU_CELLS_PER_WORKER = 256


def _oracle_cells_worker(lo_cell: int, hi_cell: int, warmup: int, steps: int, budget_s: float):
    """The oracle, as it stands, on cells [lo_cell, hi_cell) of the grid (their
    own cell ids, so their own random streams): `warmup` untimed steps, then up
    to `steps` timed ones within `budget_s`.  Returns (pairs, seconds, steps)."""
    from oracle import oracle as O

    g = I.grid_geometric(seed=0)
    m = (g.cell >= lo_cell) & (g.cell < hi_cell)
    P = O.params("geometric", dv=g.dv, seed=0)
    st = O.State(g.xi[m].copy(), g.v[m].copy(), g.cell[m].copy(), None, hi_cell)
    for s in range(warmup):
        O.step(P, st, s)
    st = O.State(g.xi[m].copy(), g.v[m].copy(), g.cell[m].copy(), None, hi_cell)
    pairs, done = 0, 0
    t0 = time.perf_counter()
    while done < steps and time.perf_counter() - t0 < budget_s:
        pairs += O.step(P, st, done % RUN_STEPS).n_pairs
        done += 1
    return pairs, time.perf_counter() - t0, done


def oracle_on_cores(warmup: int, steps: int, budget_s: float):
    """The oracle on every host core: one process per core (spawned, so safe
    after CUDA is initialised), each on its own 256 cells.  Throughput = all
    pairs / the slowest process's own timed seconds (start-up excluded)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    from oracle import oracle as O

    O.build()
    workers = max(1, min(os.cpu_count() or 1, 16384 // CPU_CELLS_PER_WORKER))
    spans = [(k * CPU_CELLS_PER_WORKER, (k + 1) * CPU_CELLS_PER_WORKER) for k in range(workers)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_cells_worker, [a for a, _ in spans], [b for _, b in spans], [warmup] * workers,
                          [steps] * workers, [budget_s] * workers))
    pairs = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    n_steps = min(r[2] for r in res)
    sample = (f"{workers} processes x {CPU_CELLS_PER_WORKER} cells of 16384 ({workers * CPU_CELLS_PER_WORKER * 256:,} "
              f"SDs), >= {n_steps} steps each from the initial state")
    return {"value": pairs / t, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
            "seconds": t, "steps": n_steps}


def cpu_baseline(seconds: float = 12.0):
    """The oracle as it stands on every host core, on a bounded sample of the grid."""
    r = oracle_on_cores(0, RUN_STEPS, seconds)
    return {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}


# -------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return None
    r = oracle_on_cores(args.warmup, args.steps, 600.0)
    value = r["value"]
    cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["seconds"] / max(1, r["steps"]) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": r["sample"]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip every extra line (same as --extras none)")
    ap.add_argument("--extras", default="all",
                    help="comma-separated extra lines to measure: " + ",".join(EXTRAS) + " (default all)")
    ap.add_argument("--serve-requests", type=int, default=200)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res))
        return
    # the oracle's timing runs before any CUDA work (no fork after CUDA init)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if res is not None:
        res["cpu_baseline"] = cpu
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
