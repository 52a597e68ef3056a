"""The grid split into pieces of whole levels with the halo exchange of
falling SDs (paper_2103_17238_gb300/shard.py), on CPU: the pieces are
stepped by the oracle here (the CUDA library steps them on a GPU, in
tests/test_gpu_shard.py), the exchange runs over the in-process loopback and
over two gloo ranks, and the pieces' state after several sedimentation and
coalescence steps equals the whole grid's run bit for bit."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2103_17238_gb300 import shard as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NZ, DZ = 6, 12, 25.0
DT = 40.0  # large drops fall several levels per step: SDs skip whole pieces


class OraclePiece:
    """A piece stepped by the oracle: its SDs with their cells in the whole
    grid (the oracle needs no cell base: it takes the grid's cell ids)."""

    def __init__(self, O, P, lo, hi, rec):
        self.O, self.P, self.lo, self.hi = O, P, lo, hi
        self.step = 0
        self.write(rec)

    def write(self, rec):
        self.rec = rec.copy()

    def read(self):
        return self.rec.copy()

    def coalesce(self, n=1):
        r = self.rec
        st = self.O.State(r["xi"].copy(), r["v"].copy(), r["cell"].copy(), None, NX * NZ)
        self.O.run(self.P, st, self.step, n)
        self.step += n
        self.rec["xi"], self.rec["v"] = st.xi, st.v

    def sediment(self):
        r = self.rec
        st = self.O.State(r["xi"].copy(), r["v"].copy(), r["cell"].copy(), None, NX * NZ)
        zeta = r["zeta"].copy()
        pr = self.O.sediment(self.P, st, NX, DZ, zeta)
        self.rec["cell"], self.rec["zeta"] = st.cell, zeta
        return pr

    def close(self):
        pass


def _initial(O, seed=3):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 40, NX * NZ)
    counts[rng.random(NX * NZ) < 0.1] = 0
    cell = np.repeat(np.arange(NX * NZ, dtype=np.int32), counts)
    n = len(cell)
    perm = rng.permutation(n)
    cell = cell[perm]
    xi = rng.integers(1, 10**8, n).astype(np.int64)
    xi[rng.random(n) < 0.03] = 0
    r = np.exp(rng.uniform(np.log(3e-6), np.log(2.5e-3), n))
    v = 4.0 / 3.0 * math.pi * r**3
    z = (cell // NX).astype(np.float64) * DZ + rng.uniform(0.0, DZ, n)
    zeta = O.zeta_of(z, cell, NX, DZ)
    return xi, v, cell, zeta


def _whole_grid(O, P, xi, v, cell, zeta, cycles):
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, NX * NZ)
    zt = zeta.copy()
    pr = 0.0
    for k in range(cycles):
        pr += O.sediment(P, st, NX, DZ, zt)
        O.step(P, st, k)
    return st, zt, pr


def _params(O):
    return O.params("geometric", dv=1e-1, dt=DT, seed=11)


def _check(rec, st, zt):
    inside = np.nonzero(st.cell >= 0)[0]
    assert np.array_equal(rec["gid"], inside)
    assert np.array_equal(rec["cell"], st.cell[inside])
    assert np.array_equal(rec["zeta"], zt[inside])
    assert np.array_equal(rec["xi"], st.xi[inside])
    assert np.array_equal(rec["v"], st.v[inside])


def test_level_ranges_and_owners():
    r = S.level_ranges(10, 3)
    assert r == [(0, 3), (3, 7), (7, 10)]
    assert [S.owner_of_level(z, r) for z in (0, 2, 3, 6, 7, 9)] == [0, 0, 1, 1, 2, 2]
    with pytest.raises(ValueError):
        S.level_ranges(2, 3)
    with pytest.raises(ValueError):
        S.owner_of_level(10, r)


@pytest.mark.parametrize("n_pieces", [1, 2, 4])
def test_pieces_in_one_process_equal_the_whole_grid(oracle_lib, n_pieces):
    O = oracle_lib
    P = _params(O)
    xi, v, cell, zeta = _initial(O)
    gid = np.arange(len(xi), dtype=np.int64)
    geom = S.Geometry(NX, NZ, DZ)
    parts = S.split_state(gid, xi, v, cell, zeta, NX, S.level_ranges(NZ, n_pieces))
    run = S.ShardedRun(geom, n_pieces, S.LoopbackComm(),
                       lambda i, lo, hi, rec: OraclePiece(O, P, lo, hi, rec)).start(parts)
    cycles = 6
    moved = 0
    for k in range(cycles):
        before = {int(g): int(c) for p in run.pieces.values() for g, c in zip(p.rec["gid"], p.rec["cell"])}
        run.sediment()
        after = run.state()
        moved += sum(1 for g, c in zip(after["gid"], after["cell"]) if before.get(int(g)) != int(c))
        run.coalesce(1)
    st, zt, pr = _whole_grid(O, P, xi, v, cell, zeta, cycles)
    _check(run.state(), st, zt)
    assert run.precipitated == pytest.approx(pr, rel=1e-12)
    assert moved > 0 and pr > 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2103_17238_gb300 import shard as S2

    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = _params(O)
    xi, v, cell, zeta = _initial(O)
    gid = np.arange(len(xi), dtype=np.int64)
    n_pieces = 3  # rank 0 holds pieces 0 and 2, rank 1 piece 1
    parts = S2.split_state(gid, xi, v, cell, zeta, NX, S2.level_ranges(NZ, n_pieces))
    run = S2.ShardedRun(S2.Geometry(NX, NZ, DZ), n_pieces, S2.TorchComm(),
                        lambda i, lo, hi, rec: OraclePiece(O, P, lo, hi, rec)).start(parts)
    for _ in range(5):
        run.sediment()
        run.coalesce(1)
    q.put((rank, run.state().tobytes(), run.precipitated, sorted(run.pieces)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_grid(oracle_lib):
    O = oracle_lib
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][3] == [0, 2] and out[1][3] == [1]
    rec = np.concatenate([np.frombuffer(o[1], S.RECORD) for o in out])
    rec = rec[np.argsort(rec["gid"])]
    P = _params(O)
    xi, v, cell, zeta = _initial(O)
    st, zt, pr = _whole_grid(O, P, xi, v, cell, zeta, 5)
    _check(rec, st, zt)
    assert out[0][2] + out[1][2] == pytest.approx(pr, rel=1e-12)
