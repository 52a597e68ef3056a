"""The oracle on several host cores, for parity checks at full size.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).  Cells and independent runs do
not interact within a coalescence step, so the oracle's result for a whole
grid or ensemble is the concatenation of its results on disjoint pieces: each
piece keeps its SDs in increasing id within every cell (so their ranks, and
with them the random streams, are unchanged) and its own cell indices.  The
pieces run in processes started with ``spawn``, which is safe after CUDA has
been initialised in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def _run_piece(args):
    from oracle import oracle as O

    pkw, xi, v, cell, n_cells, s0, steps = args
    st = O.State(xi, v, cell, None, n_cells)
    O.run(O.params(**pkw), st, s0, steps)
    return st.xi, st.v


def _workers(n_tasks: int, workers: int | None) -> int:
    return max(1, min(n_tasks, workers or os.cpu_count() or 1))


def run_cells(pkw: dict, xi, v, cell, n_cells: int, s0: int, steps: int, workers: int | None = None):
    """(xi, v) after `steps` oracle steps from step index s0 of one run of
    n_cells cells (params from ``oracle.params(**pkw)``), computed by
    contiguous cell ranges in parallel.  Inputs are indexed by SD id."""
    from oracle import oracle as O

    O.build()
    xi = np.asarray(xi, np.int64)
    v = np.asarray(v, np.float64)
    cell = np.asarray(cell, np.int32)
    w = _workers(n_cells, workers)
    bounds = np.linspace(0, n_cells, w + 1).round().astype(np.int64)
    masks, tasks = [], []
    for k in range(w):
        m = (cell >= bounds[k]) & (cell < bounds[k + 1])
        masks.append(m)
        tasks.append((pkw, xi[m].copy(), v[m].copy(), cell[m].copy(), n_cells, s0, steps))
    out_xi, out_v = xi.copy(), v.copy()
    with ProcessPoolExecutor(max_workers=w, mp_context=mp.get_context("spawn")) as ex:
        for m, (a, b) in zip(masks, ex.map(_run_piece, tasks)):
            out_xi[m] = a
            out_v[m] = b
    return out_xi, out_v


def run_many(jobs, workers: int | None = None):
    """Independent runs in parallel.  jobs: list of (pkw, xi, v, cell,
    n_cells, s0, steps); returns the list of (xi, v)."""
    from oracle import oracle as O

    O.build()
    w = _workers(len(jobs), workers)
    with ProcessPoolExecutor(max_workers=w, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run_piece, jobs, chunksize=max(1, len(jobs) // (4 * w))))
