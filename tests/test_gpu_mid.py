"""The cluster path of mid-size cells (4097 to 65536 stored SDs: one
thread-block cluster of 1, 2 or 4 CTAs per cell, the sort and the pairs in
shared and distributed shared memory) against the oracle, bit for bit, and
against the multi-pass global path (tuning mid_max_sd = 0)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


# sizes at and around the cluster sizes' edges (K = 1 up to 16384, 2 up to
# 32768, 4 up to 65536), odd sizes (padded to even slots)
SIZES = [4097, 5000, 16383, 16384, 16385, 20001, 32767, 32768, 32769, 50000, 65535, 65536]


def _state(rng, sizes, dead_frac=0.05):
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cell)
    xi = np.where(rng.random(n) < 0.3, 1000, rng.integers(1, 10**9, n)).astype(np.int64)
    xi[rng.random(n) < dead_frac] = 0
    r = np.exp(rng.uniform(np.log(2e-6), np.log(2e-3), n))
    v = 4 / 3 * np.pi * r**3
    perm = rng.permutation(n)
    return xi[perm], v[perm], cell[perm]


CLUSTER = {"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "mid_max_sd": 65536}


def _run(sdm, kernel, precision, xi, v, cell, nc, dv, seed, chunks, tuning=CLUSTER):
    sdm.sdm_set_tuning(tuning)
    try:
        run = sdm.Run(sdm.make_config(kernel, precision, dv=dv, n_cells=nc, seed=seed), len(xi))
        run.set_attributes(xi, v, cell)
        for k in chunks:
            run.step(k)
        out = run.attributes()
        run.close()
    finally:
        sdm.sdm_set_tuning(None)
    return out


@pytest.mark.parametrize("kernel,precision,dv", [("golovin", "fp64", 1e2), ("geometric", "fp64", 1e-3),
                                                 ("geometric", "kfp32", 1e1), ("golovin", "fp64", 1e-4)])
def test_mid_cells_match_the_oracle(env, kernel, precision, dv):
    O, sdm, torch = env
    rng = np.random.default_rng(71)
    xi, v, cell = _state(rng, SIZES)
    nc = len(SIZES)
    gx, gv = _run(sdm, kernel, precision, xi, v, cell, nc, dv, 13, [2, 3])
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nc)
    O.run(O.params(kernel, precision, dv=dv, seed=13), st, 0, 5)
    bad = np.nonzero(gx != st.xi)[0]
    assert bad.size == 0, f"{bad.size} multiplicities differ, first at SD {bad[0]} (cell {cell[bad[0]]})"
    assert np.array_equal(gv, st.v)
    assert int((gx != xi).sum()) > 0


def test_mid_cells_mostly_dead(env):
    """Cells of 40000 and 60000 stored SDs with only a handful alive: the
    positions are dealt to the CTAs in tiny ranges, so buckets straddle
    several CTAs' ranges and pairs read entries held by other CTAs."""
    O, sdm, torch = env
    rng = np.random.default_rng(5)
    sizes = [40000, 60000, 20000, 9000]
    xi, v, cell = _state(rng, sizes, dead_frac=0.0)
    for c, alive in zip(range(4), (11, 7, 5, 3)):
        idx = np.nonzero(cell == c)[0]
        keep = rng.choice(idx, alive, replace=False)
        dead = np.setdiff1d(idx, keep)
        xi[dead] = 0
    gx, gv = _run(sdm, "golovin", "fp64", xi, v, cell, 4, 1e-6, 3, [1, 1, 1])
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, 4)
    O.run(O.params("golovin", dv=1e-6, seed=3), st, 0, 3)
    assert np.array_equal(gx, st.xi) and np.array_equal(gv, st.v)
    assert int((gx != xi).sum()) > 0


def test_cluster_path_equals_multi_pass_path(env):
    """The same ensemble-like mix through the cluster path and through the
    multi-pass path (mid_max_sd = 0): identical states bit for bit."""
    O, sdm, torch = env
    rng = np.random.default_rng(9)
    sizes = list(np.round(2.0 ** rng.uniform(12.0, 16.0, 24)).astype(int))
    xi, v, cell = _state(rng, sizes)
    nc = len(sizes)
    base = {"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2}
    a = _run(sdm, "golovin", "fp64", xi, v, cell, nc, 1e2, 21, [4, 6], {**base, "mid_max_sd": 65536})
    b = _run(sdm, "golovin", "fp64", xi, v, cell, nc, 1e2, 21, [4, 6], {**base, "mid_max_sd": 0})
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # and with the block kernel's threshold lowered, cells from 513 SDs take the cluster path
    c = _run(sdm, "golovin", "fp64", xi, v, cell, nc, 1e2, 21, [4, 6],
             {"smem_max_sd": 512, "warp_cell_max": 512, "warps_per_block": 2, "mid_max_sd": 65536})
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
