"""A column grid split into pieces of whole levels, one context per piece
(one per GPU in a multi-process run), with a halo exchange of the SDs that
fall from one piece into another.

The paper's 2-D example has drizzle sedimenting through a grid of cells.
Cells are independent within a coalescence step, so a grid can be split
into pieces; sedimentation is the only step that moves SDs between cells,
and with no flow field it moves them only downwards, so a piece sends SDs
only to the pieces below it.  Every SD carries its id in the whole run (gid)
and its cell in the whole grid; a piece keeps its SDs in increasing gid, so
the rank of an SD in its cell (which addresses its random numbers) is its
rank in the whole grid, and the library's context of a piece uses the
whole grid's cell indices for its random streams (sdm_config.cell_base).
The pieces then step exactly as the whole grid does, bit for bit.

One coupled step (sediment, then coalesce) of every piece:
  1. the piece's sedimentation step (levels counted from the grid's bottom:
     an SD falling below the piece's lowest level continues into the levels
     below, sdm_get_heights gives its new cell and height there);
  2. the halo exchange: each piece sends every SD that entered a level of
     another piece to that piece's owner (an all-gather of per-destination
     lists over the communicator: torch.distributed, any backend, or the
     in-process loopback);
  3. each piece merges the SDs it received into its own by gid and sets the
     new state (sdm_set_attributes, sdm_set_heights: heights exactly as sent);
  4. the coalescence step.
The exchange is host-staged (each piece's state makes a round trip through
host memory in step 3), which is correct by construction and simple; its
cost is the state's transfer per sedimentation step.

The stepping backend is pluggable (`LibPiece` drives the CUDA library); the
protocol itself holds no arithmetic of the method.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

RECORD = np.dtype([("gid", np.int64), ("xi", np.int64), ("v", np.float64), ("cell", np.int32),
                   ("zeta", np.float64)])


def level_ranges(nz: int, n_pieces: int) -> list[tuple[int, int]]:
    """Contiguous level ranges [lo, hi) of n_pieces pieces, piece 0 at the
    bottom, sizes differing by at most one level."""
    if n_pieces < 1 or n_pieces > nz:
        raise ValueError(f"{n_pieces} pieces for {nz} levels")
    b = np.linspace(0, nz, n_pieces + 1).round().astype(int)
    return [(int(b[i]), int(b[i + 1])) for i in range(n_pieces)]


def owner_of_level(level: int, ranges) -> int:
    for i, (lo, hi) in enumerate(ranges):
        if lo <= level < hi:
            return i
    raise ValueError(f"level {level} outside the grid")


def split_state(gid, xi, v, cell, zeta, nx: int, ranges):
    """The records of each piece (SDs inside the grid only), sorted by gid."""
    rec = np.zeros(len(gid), RECORD)
    rec["gid"], rec["xi"], rec["v"], rec["cell"], rec["zeta"] = gid, xi, v, cell, zeta
    rec = rec[np.argsort(rec["gid"], kind="stable")]
    rec = rec[rec["cell"] >= 0]
    level = rec["cell"] // nx
    return [rec[(level >= lo) & (level < hi)].copy() for lo, hi in ranges]


@dataclass
class Geometry:
    nx: int   # columns
    nz: int   # levels of the whole grid
    dz: float  # level height, m


class LibPiece:
    """One piece stepped by the CUDA library (a context whose cells are the
    piece's levels, cell_base = its first level x nx)."""

    def __init__(self, geom: Geometry, lo: int, hi: int, records, capacity: int, *, kernel="geometric",
                 precision="fp64", dv=1e3, dt=1.0, seed=0, b=1500.0):
        from paper_2103_17238_gb300 import sdm

        self.sdm = sdm
        self.geom, self.lo, self.hi = geom, lo, hi
        self.base = lo * geom.nx
        self.n_cells = (hi - lo) * geom.nx
        self.cfg = dict(kernel=kernel, precision=precision, dv=dv, dt=dt, seed=seed, b=b)
        self.capacity = int(capacity)
        self.run = sdm.Run(sdm.make_config(kernel, precision, b=b, dt=dt, dv=dv, n_cells=self.n_cells, seed=seed,
                                           cell_base=self.base), self.capacity)
        self.gid = np.zeros(0, np.int64)
        self.step = 0  # index of the next coalescence step of the whole grid
        self.write(records)

    def write(self, rec):
        """Sets the piece's state from records sorted by gid (cells of this
        piece, heights above their cells' bottoms)."""
        self.gid = rec["gid"].copy()
        if len(rec) == 0:
            return
        if len(rec) > self.capacity:
            raise ValueError(f"piece of levels [{self.lo}, {self.hi}) needs {len(rec)} SDs, capacity {self.capacity}")
        if self.run.info().step != self.step:  # was empty while the grid stepped: resume at its step
            sdm, c = self.sdm, self.cfg
            self.run.close()
            self.run = sdm.Run(sdm.make_config(c["kernel"], c["precision"], b=c["b"], dt=c["dt"], dv=c["dv"],
                                               n_cells=self.n_cells, seed=c["seed"], cell_base=self.base,
                                               step0=self.step), self.capacity)
        self.run.set_attributes(rec["xi"], rec["v"], (rec["cell"] - self.base).astype(np.int32))
        self.sdm.sdm_set_heights(self.run.h, np.ascontiguousarray(rec["zeta"]), self.geom.nx, self.geom.dz)

    def read(self):
        """Records of every SD the piece holds: cell in the whole grid (or
        -1), height above that cell's bottom."""
        rec = np.zeros(len(self.gid), RECORD)
        if len(self.gid) == 0:
            return rec
        xi, v = self.run.attributes()
        zeta, cell = self.sdm.sdm_get_heights(self.run.h, len(self.gid))
        rec["gid"], rec["xi"], rec["v"], rec["cell"], rec["zeta"] = self.gid, xi, v, cell, zeta
        return rec

    def coalesce(self, n_steps: int = 1):
        if len(self.gid):
            self.run.step(n_steps)
        self.step += n_steps

    def sediment(self) -> float:
        return self.run.sediment() if len(self.gid) else 0.0

    def close(self):
        self.run.close()


class LoopbackComm:
    """All pieces in this process: the exchange is a reshuffle of lists."""

    rank, world = 0, 1

    def all_gather(self, obj):
        return [obj]


class TorchComm:
    """The exchange over torch.distributed (gloo, or nccl with CUDA
    devices): one all_gather_object of every rank's outgoing lists."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)

    def all_gather(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out


class ShardedRun:
    """The pieces owned by this rank (piece i lives on rank i % world) of a
    grid of geom.nz levels split into n_pieces level ranges."""

    def __init__(self, geom: Geometry, n_pieces: int, comm, make_piece):
        self.geom, self.comm = geom, comm
        self.ranges = level_ranges(geom.nz, n_pieces)
        self.mine = [i for i in range(n_pieces) if i % comm.world == comm.rank]
        self.make_piece = make_piece
        self.pieces = {}
        self.precipitated = 0.0

    def start(self, parts):
        """parts[i]: records of piece i (from split_state); only this rank's
        pieces are built."""
        for i in self.mine:
            lo, hi = self.ranges[i]
            self.pieces[i] = self.make_piece(i, lo, hi, parts[i])
        return self

    def coalesce(self, n_steps: int = 1):
        for p in self.pieces.values():
            p.coalesce(n_steps)

    def sediment(self) -> float:
        """One sedimentation step of every piece and the halo exchange;
        returns this rank's precipitated volume (sum over its pieces)."""
        nx = self.geom.nx
        outbox = {}
        keep = {}
        pr = 0.0
        for i, p in self.pieces.items():
            pr += p.sediment()
            rec = p.read()
            rec = rec[rec["cell"] >= 0]  # fallen through the grid's bottom, dead or outside: gone
            level = rec["cell"] // nx
            lo, hi = self.ranges[i]
            inside = (level >= lo) & (level < hi)
            keep[i] = rec[inside]
            for r in rec[~inside]:
                outbox.setdefault(owner_of_level(int(r["cell"] // nx), self.ranges), []).append(r)
        packed = {d: np.array(rs, RECORD) for d, rs in outbox.items()}
        arrived = {i: [] for i in self.pieces}
        for box in self.comm.all_gather(packed):
            for d, rs in box.items():
                if d in arrived:
                    arrived[d].append(rs)
        for i, p in self.pieces.items():
            rec = np.concatenate([keep[i], *arrived[i]]) if arrived[i] else keep[i]
            rec = rec[np.argsort(rec["gid"], kind="stable")]
            p.write(rec)
        self.precipitated += pr
        return pr

    def state(self):
        """Records of this rank's pieces (inside the grid), sorted by gid."""
        recs = [p.read() for p in self.pieces.values()]
        rec = np.concatenate(recs) if recs else np.zeros(0, RECORD)
        rec = rec[rec["cell"] >= 0]
        return rec[np.argsort(rec["gid"], kind="stable")]

    def close(self):
        for p in self.pieces.values():
            p.close()
