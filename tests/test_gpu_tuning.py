"""The launch tuning changes how cells are mapped to kernels, never the
result: every setting must give the oracle's state bit for bit, for cells of
every size class (and the cluster or the multi-pass path above the
shared-memory threshold), alone and in a batch; the autotuner picks one of
its candidates and caches it."""
import itertools
import json

import numpy as np
import pytest

from paper_2103_17238_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 3, 31, 33, 64, 65, 128, 129, 255, 256, 257, 511, 512, 513, 1023, 1025, 2047, 2049, 4095,
         4096, 4097, 6000]

TUNINGS = [dict(smem_max_sd=s, warp_cell_max=w, warps_per_block=k)
           for s, w, k in itertools.product((512, 1024, 2048, 4096), (0, 64, 128, 256, 512), (1, 2, 4))
           if not (w == 0 and k != 2)]
# every other setting with one launch per step, the rest with the default fusion;
# every third with the cells above the shared-memory threshold on the multi-pass
# path instead of the cluster path
for _i, _t in enumerate(TUNINGS):
    if _i % 2:
        _t["fuse_steps"] = 0
    _t["mid_max_sd"] = 0 if _i % 3 == 0 else 65536


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
    yield O, sdm, torch
    sdm.sdm_set_tuning(None)


def _state(seed):
    rng = np.random.default_rng(seed)
    cells = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(SIZES)])
    n = len(cells)
    xi = np.where(rng.random(n) < 0.3, 1000, rng.integers(1, 10**9, n)).astype(np.int64)
    xi[rng.random(n) < 0.05] = 0
    r = np.exp(rng.uniform(np.log(2e-6), np.log(2e-3), n))
    v = 4 / 3 * np.pi * r**3
    perm = rng.permutation(n)
    return xi[perm], v[perm], cells[perm]


@pytest.mark.parametrize("kernel,precision", [("geometric", "fp64"), ("golovin", "kfp32")])
def test_every_tuning_gives_the_oracle_state(env, kernel, precision):
    O, sdm, torch = env
    xi, v, cell = _state(23)
    nc, dv, seed, steps = len(SIZES), 1e3, 31, 4
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nc)
    O.run(O.params(kernel, precision, dv=dv, seed=seed), st, 0, steps)
    for t in TUNINGS:
        sdm.sdm_set_tuning(t)
        run = sdm.Run(sdm.make_config(kernel, precision, dv=dv, n_cells=nc, seed=seed), len(xi))
        run.set_attributes(xi, v, cell).step(steps)
        gx, gv = run.attributes()
        run.close()
        bad = np.nonzero(gx != st.xi)[0]
        assert bad.size == 0, f"{t}: {bad.size} multiplicities differ"
        assert np.array_equal(gv, st.v), f"{t}: volumes differ"
    sdm.sdm_set_tuning(None)


def test_autotuned_batch_equals_default(env, tmp_path):
    O, sdm, torch = env
    from paper_2103_17238_gb300 import autotune

    specs = [I.box_golovin(3000, seed=1), I.grid_geometric(side=3, sd_per_cell=256, seed=2),
             I.grid_geometric(side=2, sd_per_cell=1500, seed=3)]

    def make():
        return [sdm.Run(sdm.make_config("golovin" if g.n_cells == 1 else "geometric", dv=1e3, n_cells=g.n_cells,
                                        seed=g.seed), g.n_sd).set_attributes(g.xi, g.v, g.cell) for g in specs]

    sdm.sdm_set_tuning(None)
    ref = make()
    b = sdm.Batch(ref)
    b.step(6)
    torch.cuda.synchronize()
    b.close()

    cands = TUNINGS[::5]
    cache = str(tmp_path / "tune.json")
    probe = make()
    rep = autotune.tune(probe, steps=2, cache_path=cache, candidates=cands)
    assert not rep["cached"] and rep["best"] in cands
    assert sdm.sdm_get_tuning() == {"fuse_steps": sdm.FUSE_STEPS_DEFAULT, "mid_max_sd": sdm.MID_MAX_SD_DEFAULT,
                                    **rep["best"]}
    assert rep["ms_per_step"] <= rep["worst_ms_per_step"]
    again = autotune.tune(probe, steps=2, cache_path=cache, candidates=cands)
    assert again["cached"] and again["best"] == rep["best"]
    assert rep["key"] in json.load(open(cache))

    runs = make()
    b = sdm.Batch(runs, use_graph=True, graph_steps=3)
    b.step(6)
    torch.cuda.synchronize()
    b.close()
    for r, a in zip(runs, ref):
        x1, v1 = r.attributes()
        x2, v2 = a.attributes()
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    sdm.sdm_set_tuning(None)


@pytest.mark.parametrize("kernel,precision,fuse", [("geometric", "fp64", 7), ("golovin", "kfp32", 2),
                                                   ("geometric", "fp64", 1024)])
def test_fused_steps_give_the_oracle_state(env, kernel, precision, fuse):
    """With fusion on, every warp-per-cell cell takes up to `fuse` steps in one
    launch, the other cells one launch per step; 10 steps split as 7 + 3, 5 x 2
    and 1 x 10 must all end in the oracle's state, directly and in a graph."""
    O, sdm, torch = env
    xi, v, cell = _state(29)
    nc, dv, seed, steps = len(SIZES), 1e3, 37, 10
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nc)
    O.run(O.params(kernel, precision, dv=dv, seed=seed), st, 0, steps)
    sdm.sdm_set_tuning({"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": fuse})
    try:
        run = sdm.Run(sdm.make_config(kernel, precision, dv=dv, n_cells=nc, seed=seed), len(xi))
        run.set_attributes(xi, v, cell).step(steps)
        gx, gv = run.attributes()
        run.close()
        assert np.array_equal(gx, st.xi) and np.array_equal(gv, st.v)

        runs = [sdm.Run(sdm.make_config(kernel, precision, dv=dv, n_cells=nc, seed=seed), len(xi))
                .set_attributes(xi, v, cell) for _ in range(2)]
        b = sdm.Batch(runs, use_graph=True, graph_steps=4)
        b.step(steps)  # two graph launches of 4 steps, then 2 direct steps
        torch.cuda.synchronize()
        b.close()
        for r in runs:
            gx, gv = r.attributes()
            r.close()
            assert np.array_equal(gx, st.xi) and np.array_equal(gv, st.v)
    finally:
        sdm.sdm_set_tuning(None)


def test_fused_grid_matches_the_oracle(env):
    """A 24 x 24 grid of 256-SD cells (the shape of the flagship workload),
    30 steps in fused launches of 16 + 14."""
    O, sdm, torch = env
    g = I.grid_geometric(side=24, sd_per_cell=256, seed=5)
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, g.n_cells)
    O.run(O.params("geometric", "fp64", dv=g.dv, seed=g.seed), st, 0, 30)
    sdm.sdm_set_tuning({"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": 16})
    try:
        run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
        run.set_attributes(g.xi, g.v, g.cell).step(30)
        gx, gv = run.attributes()
        run.close()
    finally:
        sdm.sdm_set_tuning(None)
    assert np.array_equal(gx, st.xi) and np.array_equal(gv, st.v)


def test_fused_cells_that_die_out(env):
    """Cells whose SDs coalesce away inside one fused launch: pairs of xi = 1
    with p >> 1 split into a dead SD and a live one at the first step, so the
    cell has n_c = 1 for the launch's later steps; larger cells of xi = 1 halve
    their live count step after step.  Every state equals the oracle's."""
    O, sdm, torch = env
    sizes = [2, 3, 4, 5, 8, 17, 64, 255]
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cell)
    xi = np.ones(n, np.int64)
    v = np.full(n, 4 / 3 * np.pi * (50e-6) ** 3)
    nc, dv, seed, steps = len(sizes), 1e-12, 41, 12  # Golovin with a tiny dV: p far above 1
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nc)
    O.run(O.params("golovin", "fp64", dv=dv, seed=seed), st, 0, steps)
    assert (st.xi > 0).sum() < n // 2  # most SDs died
    for fuse in (0, 12, 5):
        sdm.sdm_set_tuning({"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": fuse})
        try:
            run = sdm.Run(sdm.make_config("golovin", "fp64", dv=dv, n_cells=nc, seed=seed), n)
            run.set_attributes(xi, v, cell).step(steps)
            gx, gv = run.attributes()
            run.close()
        finally:
            sdm.sdm_set_tuning(None)
        assert np.array_equal(gx, st.xi) and np.array_equal(gv, st.v), f"fuse_steps {fuse}"
