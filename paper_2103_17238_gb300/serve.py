"""Continuous-batching server of coalescence runs on one GPU.

Requests (a Golovin box or a geometric cell grid, each with its own size,
length, dt, spectrum and seed) arrive over time.  Admission is by device
memory: a request enters as soon as it has arrived and its footprint
(``sdm_footprint_bytes``) fits in what the budget has left.  Admitted runs
keep their state resident and advance together: at every tick the active set
is stepped by one fused batch (``sdm_batch_step``) of ``chunk`` steps, capped
so that no run overshoots its own length (``fuse_steps`` sets the launch
tuning's fused mode for the batches: a tick's steps of every cell of up to
512 SDs in one launch, or with 0 one launch per step; same results).  Runs that finish hand back their
dv/dlnr spectrum and final state and leave; their memory admits the next
ones.  Every run keeps its own seed and step counter, so its result is the
same alone and in any mix.

Metrics: per-run step latency (tick time on the device / steps of the tick,
each run in the tick), time in system, requests/s and aggregate
pair-updates/s over the wall time (and over the device's busy time).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from . import sdm


@dataclass
class Served:
    req: I.Request
    run: sdm.Run | None = None
    done: int = 0
    admitted_at: float | None = None
    finished_at: float | None = None
    step_latency_ms: list = field(default_factory=list)
    spectrum: np.ndarray | None = None
    xi: np.ndarray | None = None
    v: np.ndarray | None = None
    footprint: int = 0
    pairs_per_step: int = 0


def footprint(inst: I.Instance) -> int:
    largest = int(np.bincount(inst.cell, minlength=inst.n_cells).max())
    return sdm.sdm_footprint_bytes(inst.n_sd, inst.n_cells, largest)


def make_run(inst: I.Instance) -> sdm.Run:
    cfg = sdm.make_config(inst.kernel, "fp64", b=inst.b, dt=inst.dt, dv=inst.dv, n_cells=inst.n_cells,
                          seed=inst.seed)
    return sdm.Run(cfg, inst.n_sd).set_attributes(inst.xi, inst.v, inst.cell)


class Server:
    def __init__(self, budget_bytes: int, chunk: int = 20, keep_state: bool = False, use_graph: bool = False,
                 time_scale: float = 1.0, fuse_steps: int | None = None, admit_per_pass: int = 8):
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.fuse_steps = fuse_steps  # None: the process-wide tuning as it is
        self.keep_state = keep_state
        self.use_graph = use_graph
        self.time_scale = time_scale  # arrival times are divided by this
        # requests admitted per pass: a burst of arrivals is admitted a few at
        # a time, each pass overlapping a tick of the runs already admitted
        self.admit_per_pass = max(1, int(admit_per_pass))

    def _batch(self, runs):
        """A batch of the active runs; its launch plan takes the tuning of the
        moment it is built, so the fusion setting applies for that moment only."""
        if self.fuse_steps is None:
            return sdm.Batch(runs, use_graph=self.use_graph, graph_steps=self.chunk)
        prev = sdm.sdm_get_tuning()
        sdm.sdm_set_tuning({**prev, "fuse_steps": int(self.fuse_steps)})
        try:
            return sdm.Batch(runs, use_graph=self.use_graph, graph_steps=self.chunk)
        finally:
            sdm.sdm_set_tuning(prev)

    def serve(self, requests: list[I.Request]) -> dict:
        """Serves the requests (their arrival times, divided by time_scale,
        are seconds after the call).  A tick is enqueued without waiting; the
        requests that arrive meanwhile are admitted (their state uploaded on
        a stream of their own) while the tick runs on the device, and join
        at the next tick.  Tick times are CUDA-event times of the batch's
        stream."""
        import torch

        pending = [Served(r) for r in sorted(requests, key=lambda r: r.arrival)]
        for s in pending:
            s.footprint = footprint(s.req.inst)
            if s.footprint > self.budget:
                raise sdm.SdmError(sdm.SDM_EBUDGET, "serve", f"request needs {s.footprint} B > budget")
            live = np.bincount(s.req.inst.cell[s.req.inst.xi > 0], minlength=s.req.inst.n_cells)
            s.pairs_per_step = int((live // 2).sum())
        main = torch.cuda.current_stream()
        admit_stream = torch.cuda.Stream()
        active: list[Served] = []   # in the batch
        joining: list[Served] = []  # admitted, in the batch from the next tick
        finished: list[Served] = []
        used = 0
        batch = None
        members = None
        ticks = 0
        max_active = 0
        max_used = 0
        t0 = time.perf_counter()
        pair_updates = 0
        tick_ms = []

        def admit():
            nonlocal used, max_used
            now = (time.perf_counter() - t0) * self.time_scale
            took = 0
            while (pending and took < self.admit_per_pass and pending[0].req.arrival <= now
                   and used + pending[0].footprint <= self.budget):
                took += 1
                s = pending.pop(0)
                with torch.cuda.stream(admit_stream):
                    s.run = make_run(s.req.inst)  # returns after its upload has landed
                s.admitted_at = time.perf_counter() - t0
                used += s.footprint
                joining.append(s)
            max_used = max(max_used, used)

        while pending or active or joining:
            admit()
            active += joining
            joining.clear()
            if not active:
                # idle until the next arrival
                wait = pending[0].req.arrival / self.time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
                continue
            if batch is None or members != [id(s) for s in active]:
                if batch is not None:
                    batch.close()
                batch = self._batch([s.run for s in active])
                members = [id(s) for s in active]
            max_active = max(max_active, len(active))
            k = min(self.chunk, min(s.req.inst.steps - s.done for s in active))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            batch.step(k)
            e1.record(main)
            admit()  # overlaps the tick on the device
            e1.synchronize()
            dt_ms = e0.elapsed_time(e1)
            tick_ms.append(dt_ms)
            ticks += 1
            for s in active:
                s.done += k
                s.step_latency_ms.append(dt_ms / k)
                pair_updates += k * s.pairs_per_step
            still = []
            for s in active:
                if s.done >= s.req.inst.steps:
                    s.spectrum = s.run.spectrum(I.R_EDGES)
                    if self.keep_state:
                        s.xi, s.v = s.run.attributes()
                    s.finished_at = time.perf_counter() - t0
                    used -= s.footprint
                    finished.append(s)
                else:
                    still.append(s)
            if len(still) != len(active):
                batch.close()
                batch = None
                for s in active:
                    if s not in still:
                        s.run.close()
                        s.run = None
                active = still
        if batch is not None:
            batch.close()
        wall = time.perf_counter() - t0
        lat = np.concatenate([np.asarray(s.step_latency_ms) for s in finished]) if finished else np.zeros(0)
        tis = np.array([s.finished_at - s.req.arrival / self.time_scale for s in finished])
        busy = sum(tick_ms) / 1e3
        return {
            "served": finished,
            "requests": len(finished),
            "ticks": ticks,
            "max_active": max_active,
            "max_used_bytes": max_used,
            "wall_s": wall,
            "device_busy_s": busy,
            "requests_per_s": len(finished) / wall if wall > 0 else 0.0,
            "pair_updates": pair_updates,
            "pair_updates_per_s": pair_updates / wall if wall > 0 else 0.0,
            "pair_updates_per_device_s": pair_updates / busy if busy > 0 else 0.0,
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                                "p99": float(np.percentile(lat, 99)) if lat.size else None},
            "time_in_system_s": {"p50": float(np.percentile(tis, 50)) if tis.size else None,
                                 "p99": float(np.percentile(tis, 99)) if tis.size else None},
        }
