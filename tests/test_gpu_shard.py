"""The grid split into pieces of whole levels, each piece a context of the
CUDA library (sdm_config.cell_base = its first cell), with the halo exchange
of falling SDs between them (paper_2103_17238_gb300/shard.py; here all
pieces live in one process on one GPU and exchange over the loopback).
After several sedimentation and coalescence steps the pieces' state equals
the oracle's run of the whole grid bit for bit: cells, heights, xi and v."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NZ, DZ = 8, 16, 25.0
DT = 40.0


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm
    from paper_2103_17238_gb300 import shard as S

    B.build()
    O.build()
    torch.cuda.set_device(0)
    return O, sdm, S, torch


def _initial(O, seed):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 300, NX * NZ)  # warp, block and odd cells
    counts[rng.random(NX * NZ) < 0.1] = 0
    counts[5] = 6000  # a cell on the multi-pass path
    cell = np.repeat(np.arange(NX * NZ, dtype=np.int32), counts)
    n = len(cell)
    cell = cell[rng.permutation(n)]
    xi = rng.integers(1, 10**8, n).astype(np.int64)
    xi[rng.random(n) < 0.03] = 0
    r = np.exp(rng.uniform(np.log(3e-6), np.log(2.5e-3), n))
    v = 4.0 / 3.0 * math.pi * r**3
    z = (cell // NX).astype(np.float64) * DZ + rng.uniform(0.0, DZ, n)
    return xi, v, cell, O.zeta_of(z, cell, NX, DZ)


@pytest.mark.parametrize("n_pieces,kernel", [(3, "geometric"), (5, "long")])
def test_pieces_equal_the_whole_grid(env, n_pieces, kernel):
    O, sdm, S, torch = env
    xi, v, cell, zeta = _initial(O, 7 + n_pieces)
    gid = np.arange(len(xi), dtype=np.int64)
    geom = S.Geometry(NX, NZ, DZ)
    parts = S.split_state(gid, xi, v, cell, zeta, NX, S.level_ranges(NZ, n_pieces))
    run = S.ShardedRun(geom, n_pieces, S.LoopbackComm(),
                       lambda i, lo, hi, rec: S.LibPiece(geom, lo, hi, rec, len(xi), kernel=kernel, dv=1e-1,
                                                         dt=DT, seed=11)).start(parts)
    cycles = 6
    for _ in range(cycles):
        run.sediment()
        run.coalesce(1)
    got = run.state()
    precip = run.precipitated
    run.close()
    P = O.params(kernel, dv=1e-1, dt=DT, seed=11)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, NX * NZ)
    zt = zeta.copy()
    pr = 0.0
    for k in range(cycles):
        pr += O.sediment(P, st, NX, DZ, zt)
        O.step(P, st, k)
    inside = np.nonzero(st.cell >= 0)[0]
    assert np.array_equal(got["gid"], inside)
    assert np.array_equal(got["cell"], st.cell[inside])
    assert np.array_equal(got["zeta"], zt[inside])
    assert np.array_equal(got["xi"], st.xi[inside])
    assert np.array_equal(got["v"], st.v[inside])
    assert precip == pytest.approx(pr, rel=1e-12)
    assert pr > 0 and int((st.xi[inside] != xi[inside]).sum()) > 0


def test_a_piece_that_starts_empty(env):
    """The lowest piece's levels start without SDs; large drops fall into
    them from above, so that piece's context starts stepping mid-run (at the
    grid's step index, so its random streams are the grid's)."""
    O, sdm, S, torch = env
    xi, v, cell, zeta = _initial(O, 21)
    keep = cell // NX >= 6  # levels 0..5 empty
    xi, v, cell, zeta = xi[keep], v[keep], cell[keep], zeta[keep]
    gid = np.arange(len(xi), dtype=np.int64)
    geom = S.Geometry(NX, NZ, DZ)
    n_pieces = 3  # levels [0, 5), [5, 11), [11, 16)
    parts = S.split_state(gid, xi, v, cell, zeta, NX, S.level_ranges(NZ, n_pieces))
    assert len(parts[0]) == 0
    run = S.ShardedRun(geom, n_pieces, S.LoopbackComm(),
                       lambda i, lo, hi, rec: S.LibPiece(geom, lo, hi, rec, len(xi), kernel="geometric", dv=1e-1,
                                                         dt=DT, seed=5)).start(parts)
    cycles = 5
    for k in range(cycles):
        run.coalesce(1)  # coalescence first here: the empty piece counts the steps it skips
        run.sediment()
    got = run.state()
    run.close()
    P = O.params("geometric", dv=1e-1, dt=DT, seed=5)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, NX * NZ)
    zt = zeta.copy()
    for k in range(cycles):
        O.step(P, st, k)
        O.sediment(P, st, NX, DZ, zt)
    inside = np.nonzero(st.cell >= 0)[0]
    assert np.any(st.cell[inside] // NX < 5)  # SDs reached the first piece
    assert np.array_equal(got["gid"], inside)
    assert np.array_equal(got["cell"], st.cell[inside])
    assert np.array_equal(got["zeta"], zt[inside])
    assert np.array_equal(got["xi"], st.xi[inside])
    assert np.array_equal(got["v"], st.v[inside])


def test_heights_round_trip_and_emigrants(env):
    """sdm_set_heights takes heights bit for bit; after a sedimentation step
    sdm_get_heights names, for an SD that left a piece through its bottom,
    its cell in the piece below."""
    O, sdm, S, torch = env
    nx, dz = 2, 10.0
    # a piece of levels 3..4 of a 5-level grid (cells 6..9)
    run = sdm.Run(sdm.make_config("geometric", dv=1e3, dt=1.0, n_cells=4, cell_base=6), 4)
    xi = np.array([1, 1, 1, 1], np.int64)
    r = np.array([10e-6, 2e-3, 2e-3, 2e-3])  # drops of 2 mm radius fall ~9 m in 1 s
    v = 4.0 / 3.0 * math.pi * r**3
    run.set_attributes(xi, v, np.array([0, 0, 1, 3], np.int32))
    zeta = np.array([0.1 + 2.0**-40, 1.0, 9.0, 3.0])
    sdm.sdm_set_heights(run.h, zeta, nx, dz)
    z0, c0 = sdm.sdm_get_heights(run.h)
    assert np.array_equal(z0, zeta) and list(c0) == [6, 6, 7, 9]
    zz, _ = run.positions()
    assert np.array_equal(zz, np.array([30.0, 30.0, 30.0, 40.0]) + zeta)
    run.sediment()
    z1, c1 = sdm.sdm_get_heights(run.h)
    _, local = run.positions(want_z=False)
    # SD 1 (at 1 m above level 3's bottom) falls into level 2: cell 4, below the piece
    assert c1[1] == 4 and local[1] == -1 and 0.0 <= z1[1] < dz
    assert c1[2] == 7 and local[2] == 1  # 9 m - 8.99 m: still in level 3
    assert c1[0] == 6 and local[0] == 0
    run.close()
