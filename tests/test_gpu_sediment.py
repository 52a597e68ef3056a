"""Parity of the sedimentation step with the oracle: cells, heights, xi and v
bit for bit after every step, sedimentation and coalescence steps
interleaved, on ragged columns (empty and odd cells, dead SDs, SDs already
outside the domain) and on the full 128 x 128 grid; the precipitated volume
within its summation bound; errors and the batch's layout check."""
import math

import numpy as np
import pytest

from paper_2103_17238_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U = 2.0**-53


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm

    B.build()
    O.build()
    torch.cuda.set_device(0)
    return O, sdm, torch


def _column_state(rng, nx, nz, dz, max_per_cell=300):
    sizes = rng.integers(0, max_per_cell, nx * nz)
    sizes[rng.random(nx * nz) < 0.1] = 0
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n_out = 37
    cell = np.concatenate([cell, np.full(n_out, -1, np.int32)])
    n = len(cell)
    r = np.exp(rng.uniform(np.log(3e-6), np.log(3e-3), n))
    v = 4.0 / 3.0 * np.pi * r**3
    xi = rng.integers(1, 10**9, n).astype(np.int64)
    xi[rng.random(n) < 0.03] = 0
    zeta0 = rng.uniform(0.0, dz, n)
    z = np.where(cell >= 0, (cell // nx).astype(np.float64) * dz + zeta0, 0.0)
    # inside its level (the sum can round up to the level's top)
    top = (cell // nx + 1).astype(np.float64) * dz
    z = np.where((cell >= 0) & (z >= top), np.nextafter(top, 0.0), z)
    lvl0 = np.nonzero((cell >= 0) & (cell < nx))[0][:3]
    z[lvl0] = -0.0  # a signed zero at the domain bottom
    perm = rng.permutation(n)
    return xi[perm], v[perm], cell[perm], z[perm]


def _compare(O, run, st, zeta, nx, dz, what):
    gx, gv = run.attributes()
    gz, gc = run.positions()
    assert np.array_equal(gc, st.cell), f"{what}: cells differ at {np.nonzero(gc != st.cell)[0][:5]}"
    inside = st.cell >= 0
    want_z = O.z_of(zeta[inside], st.cell[inside], nx, dz)
    assert np.array_equal(gz[inside], want_z), f"{what}: heights differ"
    assert np.all(gz[~inside] == 0.0)
    assert np.array_equal(gx, st.xi), f"{what}: multiplicities differ"
    assert np.array_equal(gv, st.v), f"{what}: volumes differ"


@pytest.mark.parametrize("dt,rounds", [(5.0, 10), (200.0, 5)])
def test_sedimentation_and_coalescence_interleaved(env, dt, rounds):
    O, sdm, torch = env
    rng = np.random.default_rng(int(dt))
    nx, nz, dz = 4, 6, 10.0
    xi, v, cell, z = _column_state(rng, nx, nz, dz)
    n_cells = nx * nz
    cfg = sdm.make_config("geometric", "fp64", dt=dt, dv=1e3, n_cells=n_cells, seed=7)
    run = sdm.Run(cfg, len(xi)).set_attributes(xi, v, cell).set_positions(z, nx, dz)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, n_cells)
    zeta = np.where(cell >= 0, O.zeta_of(z, np.maximum(cell, 0), nx, dz), 0.0)
    P = O.params("geometric", dt=dt, dv=1e3, seed=7)
    _compare(O, run, st, zeta, nx, dz, "initial")
    for t in range(rounds):
        got_p = run.sediment()
        want_p = O.sediment(P, st, nx, dz, zeta)
        n_left = int((st.cell < 0).sum())
        assert math.isclose(got_p, want_p, rel_tol=max(1e-12, 2 * len(xi) * U), abs_tol=0.0)
        _compare(O, run, st, zeta, nx, dz, f"after sedimentation {t}")
        run.step(1)
        O.step(P, st, t)
        _compare(O, run, st, zeta, nx, dz, f"after coalescence {t}")
    assert n_left > 37 + int((xi == 0).sum())  # SDs fell through the bottom
    assert int((st.xi != xi).sum()) > 0        # and collided
    # the spectrum counts only the SDs inside
    got = run.spectrum(I.R_EDGES)
    want = O.spectrum(P, st, I.R_EDGES)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    run.close()


def test_launch_plan_follows_the_layout(env):
    """A context's own launch plan is rebuilt on the device after each
    sedimentation step while its cells stay in the shared-memory classes.
    Here SDs of the second level land in the bottom one, so its cells grow
    past 4096 SDs (the plan goes back to the host, the cells to the cluster
    path), and the tuning changes between steps (also back to the host);
    every step against the oracle."""
    O, sdm, torch = env
    rng = np.random.default_rng(31)
    nx, nz, dz, dt = 2, 4, 10.0, 40.0
    sizes = [3800, 3800, 2000, 2000, 500, 500, 500, 500]
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cell)
    level = cell // nx
    r = np.where(level == 1, rng.uniform(45e-6, 55e-6, n), rng.uniform(5e-6, 15e-6, n))
    v = 4.0 / 3.0 * np.pi * r**3
    xi = rng.integers(1, 10**6, n).astype(np.int64)
    z = level.astype(np.float64) * dz + rng.uniform(0.0, dz, n)
    perm = rng.permutation(n)
    xi, v, cell, z = xi[perm], v[perm], cell[perm], z[perm]
    cfg = sdm.make_config("geometric", "fp64", dt=dt, dv=1e6, n_cells=nx * nz, seed=3)
    P = O.params("geometric", dt=dt, dv=1e6, seed=3)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nx * nz)
    zeta = O.zeta_of(z, cell, nx, dz)
    sdm.sdm_set_tuning(None)
    try:
        run = sdm.Run(cfg, n).set_attributes(xi, v, cell).set_positions(z, nx, dz)
        run.step(1)  # the plan: shared-memory classes only
        O.step(P, st, 0)
        for t in range(1, 5):
            if t == 3:
                sdm.sdm_set_tuning({"smem_max_sd": 1024, "warp_cell_max": 256, "warps_per_block": 2})
            run.sediment()
            O.sediment(P, st, nx, dz, zeta)
            _compare(O, run, st, zeta, nx, dz, f"after sedimentation {t}")
            run.step(1)
            O.step(P, st, t)
            _compare(O, run, st, zeta, nx, dz, f"after coalescence {t}")
            if t == 1:
                counts = np.bincount(st.cell[st.cell >= 0], minlength=nx * nz)
                assert counts[:nx].max() > 4096, counts  # a bottom cell left the shared-memory classes
        run.close()
    finally:
        sdm.sdm_set_tuning(None)


def test_full_grid_sedimentation(env):
    """The 128 x 128 x 256 grid as a 128-column, 128-level domain of 10 m
    levels: two rounds of sedimentation and coalescence, every SD compared."""
    O, sdm, torch = env
    g = I.grid_geometric(seed=0)
    nx, dz = 128, 10.0
    rng = np.random.default_rng(2)
    z = (g.cell // nx).astype(np.float64) * dz + rng.uniform(0.0, 0.05, g.n_sd)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, dt=20.0, n_cells=g.n_cells, seed=0), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell).set_positions(z, nx, dz)
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, g.n_cells)
    zeta = O.zeta_of(z, g.cell, nx, dz)
    P = O.params("geometric", dv=g.dv, dt=20.0, seed=0)
    for t in range(2):
        run.sediment()
        O.sediment(P, st, nx, dz, zeta)
        run.step(1)
        O.step(P, st, t)
    _compare(O, run, st, zeta, nx, dz, "full grid")
    assert int((st.cell != g.cell).sum()) > 1000
    run.close()


def test_errors_and_state(env):
    O, sdm, torch = env
    g = I.grid_geometric(side=2, sd_per_cell=64, seed=1)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=4), g.n_sd).set_attributes(g.xi, g.v, g.cell)
    with pytest.raises(sdm.SdmError) as e:
        run.sediment()
    assert e.value.status == sdm.SDM_ESTATE
    z = (g.cell // 2).astype(np.float64) * 10.0 + 1.0
    with pytest.raises(sdm.SdmError) as e:
        run.set_positions(z, 3, 10.0)              # 3 does not divide 4 cells
    assert e.value.status == sdm.SDM_EINVAL
    bad = z.copy()
    bad[17] += 10.0                                # in the level above its cell
    with pytest.raises(sdm.SdmError) as e:
        run.set_positions(bad, 2, 10.0)
    assert e.value.status == sdm.SDM_EINVAL and "SD 17" in str(e.value)
    run.set_positions(z, 2, 10.0)
    run.sediment()
    run.set_attributes(g.xi, g.v, g.cell)          # new attributes drop the positions
    with pytest.raises(sdm.SdmError) as e:
        run.sediment()
    assert e.value.status == sdm.SDM_ESTATE
    _, cells = run.positions(want_z=False)         # cells need no positions
    assert np.array_equal(cells, g.cell)
    run.close()


def test_batch_refuses_a_moved_context(env):
    O, sdm, torch = env
    g = I.grid_geometric(side=2, sd_per_cell=64, seed=1)
    runs = [sdm.Run(sdm.make_config("geometric", dv=g.dv, dt=50.0, n_cells=4, seed=s), g.n_sd)
            .set_attributes(g.xi, g.v, g.cell) for s in range(2)]
    z = (g.cell // 2).astype(np.float64) * 10.0 + 0.5
    runs[1].set_positions(z, 2, 10.0)
    batch = sdm.Batch(runs)
    batch.step(2)
    runs[1].sediment()
    with pytest.raises(sdm.SdmError) as e:
        batch.step(1)
    assert e.value.status == sdm.SDM_ESTATE
    batch.close()
    batch = sdm.Batch(runs)                        # a new batch takes the new layout
    batch.step(1)
    torch.cuda.synchronize()
    batch.close()
    for r in runs:
        r.close()
