"""Parity of the CUDA path (through the C ABI) with the oracle.

Multiplicities must match bit for bit; volumes within 1e-12 relative (the
design reproduces every binary64 operation, so equality is asserted and the
relative error reported on failure).  The spectrum sums in a different order
than the oracle, so it is compared within the summation bound
2 n u (u = 2^-53, n summands), floor 1e-12.
"""
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


def _assert_same(xi_gpu, v_gpu, st, what=""):
    bad = np.nonzero(xi_gpu != st.xi)[0]
    assert bad.size == 0, f"{what}: {bad.size} multiplicities differ, first at SD {bad[0]}"
    rel = np.abs(v_gpu - st.v) / np.abs(st.v)
    assert rel.max() <= 1e-12, f"{what}: volume rel err {rel.max()}"
    assert np.array_equal(v_gpu, st.v), f"{what}: volumes differ by at most {rel.max():.3g} relative"


def _gpu_run(sdm, kernel, precision, xi, v, cell, n_cells, dv, seed, steps, dt=1.0, b=1500.0, chunks=None,
             step0=0):
    run = sdm.Run(sdm.make_config(kernel, precision, b=b, dt=dt, dv=dv, n_cells=n_cells, seed=seed,
                                  step0=step0), len(xi))
    run.set_attributes(xi, v, cell)
    for k in (chunks or [steps]):
        run.step(k)
    return run


def _oracle_run(O, kernel, precision, xi, v, cell, n_cells, dv, seed, steps, dt=1.0, b=1500.0, s0=0):
    st = O.State(np.array(xi, np.int64), np.array(v, np.float64), np.array(cell, np.int32), None, n_cells)
    O.run(O.params(kernel, precision, b=b, dt=dt, dv=dv, seed=seed), st, s0, steps)
    return st


def test_box_golovin_full_run(env):
    """The paper's Golovin box at n_sd = 2^12: all 3600 steps, bit for bit."""
    O, sdm, torch = env
    g = I.box_golovin(2**12, seed=0)
    run = _gpu_run(sdm, "golovin", "fp64", g.xi, g.v, g.cell, 1, g.dv, 0, 3600, chunks=[1200, 1200, 1200])
    xi, v = run.attributes()
    st = _oracle_run(O, "golovin", "fp64", g.xi, g.v, g.cell, 1, g.dv, 0, 3600)
    _assert_same(xi, v, st, "box 3600 steps")
    assert run.info().step == 3600
    got = run.spectrum(I.R_EDGES)
    want = O.spectrum(O.params("golovin", dv=g.dv), st, I.R_EDGES)
    assert np.allclose(got, want, rtol=max(1e-12, 2 * g.n_sd * U), atol=0)
    run.close()


@pytest.mark.parametrize("kernel", ["golovin", "geometric", "long"])
@pytest.mark.parametrize("precision", ["fp64", "kfp32"])
def test_grid(env, kernel, precision):
    O, sdm, torch = env
    g = I.grid_geometric(side=8, sd_per_cell=256, seed=5)
    dv = g.dv if kernel == "geometric" else 1e-2  # Golovin collisions frequent enough
    run = _gpu_run(sdm, kernel, precision, g.xi, g.v, g.cell, g.n_cells, dv, 5, 40, chunks=[1, 13, 26])
    xi, v = run.attributes()
    st = _oracle_run(O, kernel, precision, g.xi, g.v, g.cell, g.n_cells, dv, 5, 40)
    _assert_same(xi, v, st, f"grid {kernel} {precision}")
    assert int((xi != g.xi).sum()) > 0  # collisions happened
    per_cell = run.spectrum(I.R_EDGES, per_cell=True)
    want = O.spectrum(O.params(kernel, precision, dv=dv), st, I.R_EDGES, per_cell=True)
    assert np.allclose(per_cell, want, rtol=max(1e-12, 2 * 256 * U), atol=0)
    run.close()


@pytest.mark.parametrize("precision", ["fp64", "kfp32"])
def test_grid_long_run(env, precision):
    """600 steps of an 8 x 8 grid of the benchmark's cells: late in the run
    the spectrum is broad, many pairs have p > 1 and their p - u falls near
    an integer, so the binary32 filter decides close to its interval bound
    and the exact path takes the pairs it leaves.  Bit for bit throughout."""
    O, sdm, torch = env
    g = I.grid_geometric(side=8, sd_per_cell=256, seed=0)
    run = _gpu_run(sdm, "geometric", precision, g.xi, g.v, g.cell, g.n_cells, g.dv, 0, 600, chunks=[150, 450])
    xi, v = run.attributes()
    st = _oracle_run(O, "geometric", precision, g.xi, g.v, g.cell, g.n_cells, g.dv, 0, 600)
    _assert_same(xi, v, st, f"grid 600 steps {precision}")
    assert int((xi != g.xi).sum()) > g.n_sd // 2  # most SDs collided
    run.close()


RAGGED = [0, 1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 513, 1000, 2047, 2049,
          4095, 4096, 4097, 5000, 9001, 20001]


def _ragged_state(rng, sizes, p_scale):
    cells = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cells)
    # mixed multiplicities: equal runs (splits), wide spread (caps), some dead
    xi = np.where(rng.random(n) < 0.3, 1000, rng.integers(1, 10**9, n)).astype(np.int64)
    xi[rng.random(n) < 0.05] = 0
    xi[rng.random(n) < 0.05] = 1
    r = np.exp(rng.uniform(np.log(2e-6), np.log(2e-3), n))
    v = 4 / 3 * np.pi * r**3
    perm = rng.permutation(n)  # unsorted cell order exercises the stable layout
    return xi[perm], v[perm], cells[perm]


@pytest.mark.parametrize("kernel,precision,dv", [("golovin", "fp64", 1e3), ("geometric", "fp64", 1e3),
                                                 ("geometric", "kfp32", 1e3), ("golovin", "fp64", 1e-3),
                                                 ("geometric", "fp64", 1e-4), ("long", "fp64", 1e3),
                                                 ("long", "kfp32", 1e-4)])
def test_ragged_cells_every_class(env, kernel, precision, dv):
    """Every shared-memory size class, its edges, empty/odd/tiny cells and the
    big-cell path; dead SDs, equal and extreme multiplicities; unsorted
    input.  Small dv drives p >> 1 (gamma > 1 and the cap)."""
    O, sdm, torch = env
    rng = np.random.default_rng(17)
    xi, v, cell = _ragged_state(rng, RAGGED, dv)
    nc = len(RAGGED)
    run = _gpu_run(sdm, kernel, precision, xi, v, cell, nc, dv, 9, 12, chunks=[5, 7])
    gx, gv = run.attributes()
    st = _oracle_run(O, kernel, precision, xi, v, cell, nc, dv, 9, 12)
    _assert_same(gx, gv, st, f"ragged {kernel} {precision} dv={dv}")
    assert int((gx != xi).sum()) > 0
    run.close()


@pytest.mark.parametrize("kernel", ["golovin", "geometric", "long"])
@pytest.mark.parametrize("precision", ["fp64", "kfp32"])
def test_probability_sweep(env, kernel, precision):
    """p from ~1e-3 to ~1e3 (dV over six decades): gamma = 0, 1, several,
    capped at floor(xi_j / xi_k), and counts whose p - u lies near an
    integer, across the 64/128/256-SD warp classes and a 512-SD block class."""
    O, sdm, torch = env
    rng = np.random.default_rng(99)
    sizes = [64, 128, 256, 512, 200, 90]
    for dv in (1e3, 1e1, 1e-1, 1e-3):
        n = sum(sizes)
        cell = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
        xi = rng.integers(1, 10**7, n).astype(np.int64)
        xi[rng.random(n) < 0.2] = 5000
        r = np.exp(rng.uniform(np.log(3e-6), np.log(1e-3), n))
        v = 4 / 3 * np.pi * r**3
        run = _gpu_run(sdm, kernel, precision, xi, v, cell, len(sizes), dv, 123, 8, chunks=[3, 5])
        gx, gv = run.attributes()
        st = _oracle_run(O, kernel, precision, xi, v, cell, len(sizes), dv, 123, 8)
        _assert_same(gx, gv, st, f"sweep {kernel} {precision} dv={dv}")
        run.close()


def test_terminal_velocity_regime_edges(env):
    """Radii within a few ulp of the Rogers-Yau boundaries, where the binary32
    filter must abstain."""
    O, sdm, torch = env
    rng = np.random.default_rng(3)
    r = np.concatenate([40e-6 * (1 + rng.uniform(-1e-6, 1e-6, 600)), 600e-6 * (1 + rng.uniform(-1e-6, 1e-6, 600)),
                        np.exp(rng.uniform(np.log(1e-6), np.log(1e-3), 848))])
    v = 4 / 3 * np.pi * r**3
    n = len(v)
    xi = rng.integers(1, 10**6, n).astype(np.int64)
    cell = np.repeat(np.arange(8, dtype=np.int32), n // 8)
    for prec in ("fp64", "kfp32"):
        run = _gpu_run(sdm, "geometric", prec, xi, v, cell, 8, 1e-3, 21, 6)
        gx, gv = run.attributes()
        st = _oracle_run(O, "geometric", prec, xi, v, cell, 8, 1e-3, 21, 6)
        _assert_same(gx, gv, st, f"regime edges {prec}")
        run.close()


@pytest.mark.parametrize("precision", ["fp64", "kfp32"])
def test_long_efficiency_edges(env, precision):
    """Long's efficiency where the binary32 filter must abstain or is near
    its bound: collector radii within a few ulp of 50 um (the switch to
    E = 1), collected radii near 3 um (1 - c2 / r cancels to the 1e-3
    floor), near-equal radii (the speed difference cancels), across the
    warp, block and multi-pass size classes."""
    O, sdm, torch = env
    rng = np.random.default_rng(31)
    n_each = 700
    r = np.concatenate([
        50e-6 * (1 + rng.uniform(-1e-6, 1e-6, n_each)),
        3e-6 * (1 + rng.uniform(-1e-3, 1e-3, n_each)),
        30e-6 * (1 + rng.uniform(-1e-7, 1e-7, n_each)),
        np.exp(rng.uniform(np.log(1e-6), np.log(2e-4), 3 * n_each)),
    ])
    v = 4 / 3 * np.pi * r**3
    n = len(v)
    xi = rng.integers(1, 10**6, n).astype(np.int64)
    sizes = [64, 200, 256, 500, 1000, 2000]
    cell = np.concatenate([np.full(k, c, np.int32) for c, k in enumerate(sizes)])
    cell = np.concatenate([cell, np.full(n - len(cell), len(sizes), np.int32)])  # one 5200-SD cell
    perm = rng.permutation(n)
    xi, v, cell = xi[perm], v[perm], cell[perm]
    for dv in (1e-2, 1e-5):
        run = _gpu_run(sdm, "long", precision, xi, v, cell, len(sizes) + 1, dv, 77, 6, chunks=[2, 4])
        gx, gv = run.attributes()
        st = _oracle_run(O, "long", precision, xi, v, cell, len(sizes) + 1, dv, 77, 6)
        _assert_same(gx, gv, st, f"Long edges {precision} dv={dv}")
        assert int((gx != xi).sum()) > 0
        run.close()


def test_spectrum_bin_edges(env):
    """Radii on, just below and just above every bin edge (relative 1e-15 ..
    1e-5): the binary32 radius must defer to the exact one there, so every SD
    lands in the bin of the definition."""
    O, sdm, torch = env
    e = I.R_EDGES
    rs = []
    for x in e:
        for d in (0.0, 1e-15, -1e-15, 1e-12, -1e-12, 1e-9, -1e-9, 1e-6, -1e-6, 6e-5, -6e-5):
            rs.append(x * (1.0 + d))
    r = np.array(rs)
    v = 4.0 / 3.0 * np.pi * r**3
    n = len(v) + (len(v) % 2)
    v = np.resize(v, n)
    xi = np.arange(1, n + 1, dtype=np.int64) * 1000
    cell = (np.arange(n) % 4).astype(np.int32)
    run = sdm.Run(sdm.make_config("golovin", dv=1e3, n_cells=4), n).set_attributes(xi, v, cell)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, 4)
    P = O.params("golovin", dv=1e3)
    got = run.spectrum(e, per_cell=True)
    want = O.spectrum(P, st, e, per_cell=True)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    assert np.array_equal(got > 0, want > 0)
    # the total over cells (up to 32 bins: the atomic-free kernel, whose
    # fixed summation order repeats bit for bit), and with 63 bins
    got_t = run.spectrum(e)
    want_t = O.spectrum(P, st, e)
    assert np.allclose(got_t, want_t, rtol=1e-12, atol=0)
    assert np.array_equal(got_t > 0, want_t > 0)
    assert np.array_equal(run.spectrum(e), got_t)
    e64 = np.logspace(np.log10(10.0e-6), np.log10(5.0e-3), 64)
    assert np.allclose(run.spectrum(e64), O.spectrum(P, st, e64), rtol=1e-12, atol=0)
    run.close()


def test_big_cell_path(env):
    O, sdm, torch = env
    g = I.box_golovin(2**17 + 6, seed=4)
    run = _gpu_run(sdm, "golovin", "fp64", g.xi, g.v, g.cell, 1, 1e2, 4, 6, chunks=[2, 4])
    gx, gv = run.attributes()
    st = _oracle_run(O, "golovin", "fp64", g.xi, g.v, g.cell, 1, 1e2, 4, 6)
    _assert_same(gx, gv, st, "big cell")
    run.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_large_single_cell_full_size(env, seed):
    """2^20 SDs in one cell (the single-large-cell workload, two of its
    ensemble seeds), 12 steps through the multi-pass path, batched as the
    benchmark steps it."""
    O, sdm, torch = env
    g = I.box_golovin(2**20, seed=seed)
    run = sdm.Run(sdm.make_config("golovin", "fp64", dv=g.dv, seed=seed), g.n_sd).set_attributes(g.xi, g.v, g.cell)
    batch = sdm.Batch([run])
    batch.step(5)
    batch.step(7)
    torch.cuda.synchronize()
    batch.close()
    gx, gv = run.attributes()
    st = _oracle_run(O, "golovin", "fp64", g.xi, g.v, g.cell, 1, g.dv, seed, 12)
    _assert_same(gx, gv, st, f"2^20 cell seed {seed}")
    assert int((gx != g.xi).sum()) > 0
    run.close()


def test_ensemble_members_match_the_oracle(env):
    """Every 8th member of the 1024-box ensemble (n_sd = 2^U(8,16): warp,
    block and multi-pass cells side by side), 20 steps as one batch replayed
    from a CUDA graph, each member against the oracle run alone."""
    O, sdm, torch = env
    insts = I.batched_ensemble(steps=20)[::8]
    runs = [sdm.Run(sdm.make_config("golovin", "fp64", dv=t.dv, seed=t.seed), t.n_sd).set_attributes(t.xi, t.v, t.cell)
            for t in insts]
    assert min(t.n_sd for t in insts) < 512 and max(t.n_sd for t in insts) > 4096
    batch = sdm.Batch(runs, use_graph=True, graph_steps=5)
    batch.step(20)
    torch.cuda.synchronize()
    batch.close()
    for t, r in zip(insts, runs):
        gx, gv = r.attributes()
        st = _oracle_run(O, "golovin", "fp64", t.xi, t.v, t.cell, 1, t.dv, t.seed, 20)
        _assert_same(gx, gv, st, f"ensemble member n_sd={t.n_sd} seed={t.seed}")
        r.close()


def test_full_grid(env):
    """The 128 x 128 x 256 geometric grid (4.19M SDs) in the launch
    configuration the benchmark times (one step per call), 12 steps, every
    SD compared."""
    O, sdm, torch = env
    g = I.grid_geometric(seed=0)
    run = _gpu_run(sdm, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 0, 12, chunks=[1] * 12)
    gx, gv = run.attributes()
    st = _oracle_run(O, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 0, 12)
    _assert_same(gx, gv, st, "full grid")
    got = run.spectrum(I.R_EDGES)
    want = O.spectrum(O.params("geometric", dv=g.dv), st, I.R_EDGES)
    assert np.allclose(got, want, rtol=max(1e-12, 2 * g.n_sd * U), atol=0)
    run.close()
    # the same 12 steps in fused launches (12, then 5 + 5 + 2), every SD compared
    for fuse, chunks in ((12, [12]), (5, [12])):
        sdm.sdm_set_tuning({"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2, "fuse_steps": fuse})
        try:
            run = _gpu_run(sdm, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 0, 12, chunks=chunks)
        finally:
            sdm.sdm_set_tuning(None)
        gx, gv = run.attributes()
        run.close()
        _assert_same(gx, gv, st, f"full grid, fused by {fuse}")


def test_sort_keys_sharing_their_top_bits(env):
    """Cells of the full grid (seed 0, step 0) in which two keys share their
    top 24 bits, order against their ranks and fall in different pairs
    (golden/sort_word_ties.txt, from the oracle's keys).  dV = 1e-3 makes
    p >> 1, so every pair collides and a wrong pairing shows in the state."""
    import os

    O, sdm, torch = env
    path = os.path.join(os.path.dirname(__file__), "golden", "sort_word_ties.txt")
    cells = sorted({int(line.split()[0]) for line in open(path) if not line.startswith("#")})
    g = I.grid_geometric(seed=0)
    keep = np.isin(g.cell, cells)
    xi, v, cell = g.xi[keep], g.v[keep], g.cell[keep]
    assert len(xi) == 256 * len(cells)
    run = _gpu_run(sdm, "geometric", "fp64", xi, v, cell, g.n_cells, 1e-3, 0, 1)
    gx, gv = run.attributes()
    st = _oracle_run(O, "geometric", "fp64", xi, v, cell, g.n_cells, 1e-3, 0, 1)
    _assert_same(gx, gv, st, "24-bit key ties")
    assert int((gx != xi).sum()) > 0.9 * len(xi)
    run.close()


@pytest.mark.parametrize("kernel,precision", [("geometric", "fp64"), ("golovin", "fp64"), ("geometric", "kfp32")])
def test_extreme_multiplicities(env, kernel, precision):
    """Multiplicities across the int64 range (1, 2^31 - 1, 2^32 + 1, 2^53 + 1,
    2^62, ...): the conversions past 32 and 53 bits, the cap with g xi_k past
    2^64, and large products in the update, with p from small to huge."""
    O, sdm, torch = env
    rng = np.random.default_rng(41)
    sizes = [2, 3, 64, 65, 255, 256, 511, 700, 5000]
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cell)
    choices = np.array([1, 2, 3, 1000, 2**31 - 1, 2**32 + 1, 2**40 + 7, 2**53 + 1, 2**60, 2**62, 2**62 + 12345],
                       dtype=np.int64)
    xi = choices[rng.integers(0, len(choices), n)]
    wide = rng.random(n) < 0.3
    xi[wide] = rng.integers(1, 2**62, int(wide.sum()))
    r = np.exp(rng.uniform(np.log(1e-6), np.log(3e-3), n))
    v = 4 / 3 * np.pi * r**3
    perm = rng.permutation(n)
    xi, v, cell = xi[perm], v[perm], cell[perm]
    for dv in (1e30, 1e6, 1e-6):
        run = _gpu_run(sdm, kernel, precision, xi, v, cell, len(sizes), dv, 5, 3)
        gx, gv = run.attributes()
        st = _oracle_run(O, kernel, precision, xi, v, cell, len(sizes), dv, 5, 3)
        _assert_same(gx, gv, st, f"extreme xi, dv={dv}")
        got = run.spectrum(I.R_EDGES)
        want = O.spectrum(O.params(kernel, precision, dv=dv), st, I.R_EDGES)
        assert np.allclose(got, want, rtol=1e-12, atol=0)
        run.close()


def test_device_inputs_and_outputs(env):
    O, sdm, torch = env
    g = I.grid_geometric(side=4, sd_per_cell=200, seed=8)
    dev = torch.device("cuda", 0)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=8), g.n_sd)
    run.set_attributes(torch.from_numpy(g.xi).to(dev), torch.from_numpy(g.v).to(dev),
                       torch.from_numpy(g.cell).to(dev))
    run.step(7)
    xi_d = torch.empty(g.n_sd, dtype=torch.int64, device=dev)
    v_d = torch.empty(g.n_sd, dtype=torch.float64, device=dev)
    sdm.sdm_get_attributes(run.h, xi=xi_d, volume=v_d)
    spec_d = torch.empty(len(I.R_EDGES) - 1, dtype=torch.float64, device=dev)
    run.spectrum(I.R_EDGES, out=spec_d)
    torch.cuda.synchronize()
    st = _oracle_run(O, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 8, 7)
    _assert_same(xi_d.cpu().numpy(), v_d.cpu().numpy(), st, "device io")
    want = O.spectrum(O.params("geometric", dv=g.dv), st, I.R_EDGES)
    assert np.allclose(spec_d.cpu().numpy(), want, rtol=1e-12, atol=0)
    run.close()


def test_resume_bit_exact(env):
    O, sdm, torch = env
    g = I.grid_geometric(side=4, sd_per_cell=256, seed=2)
    straight = _gpu_run(sdm, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 2, 30)
    a = _gpu_run(sdm, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 2, 11)
    xi, v = a.attributes()
    b = _gpu_run(sdm, "geometric", "fp64", xi, v, g.cell, g.n_cells, g.dv, 2, 19, step0=11)
    x1, v1 = straight.attributes()
    x2, v2 = b.attributes()
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    for r in (straight, a, b):
        r.close()


def test_new_attributes_keep_or_rebuild_the_plan(env):
    """set_attributes on a stepped context: a new state with the same cell
    layout (the launch plan is kept) and then one with another layout (the
    plan is rebuilt) continue exactly like fresh contexts started at those
    steps, and like the oracle."""
    O, sdm, torch = env
    g = I.grid_geometric(side=4, sd_per_cell=256, seed=3)
    xi2, v2 = g.xi // 3 + 1, g.v * 1.7
    rng = np.random.default_rng(5)
    xi3, v3, c3 = _ragged_state(rng, RAGGED[:16], 1e3)
    run = _gpu_run(sdm, "geometric", "fp64", g.xi, g.v, g.cell, g.n_cells, g.dv, 3, 4)
    run.set_attributes(xi2, v2, g.cell).step(5)
    ref = _gpu_run(sdm, "geometric", "fp64", xi2, v2, g.cell, g.n_cells, g.dv, 3, 5, step0=4)
    for a, b in zip(run.attributes(), ref.attributes()):
        assert np.array_equal(a, b)
    run.set_attributes(xi3, v3, c3).step(3)
    gx, gv = run.attributes()
    st = _oracle_run(O, "geometric", "fp64", xi3, v3, c3, g.n_cells, g.dv, 3, 3, s0=9)
    _assert_same(gx, gv, st, "new layout after 9 steps")
    assert run.info().step == 12
    for r in (run, ref):
        r.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(env, use_graph):
    """Runs of different kernels, sizes, dt and dv stepped together give the
    same state as each stepped alone."""
    O, sdm, torch = env
    specs = [("golovin", I.box_golovin(3000, seed=1), 1.0, 1e3),
             ("geometric", I.grid_geometric(side=3, sd_per_cell=256, seed=2), 2.0, 1e3),
             ("golovin", I.box_golovin(9000, seed=3), 0.5, 1e2),
             ("geometric", I.grid_geometric(side=2, sd_per_cell=64, seed=4), 1.0, 1e2),
             ("golovin", I.box_golovin(100, seed=5), 1.0, 1e-2)]
    runs, alone = [], []
    for k, g, dt, dv in specs:
        runs.append(sdm.Run(sdm.make_config(k, dt=dt, dv=dv, n_cells=g.n_cells, seed=g.seed), g.n_sd)
                    .set_attributes(g.xi, g.v, g.cell))
        alone.append(_gpu_run(sdm, k, "fp64", g.xi, g.v, g.cell, g.n_cells, dv, g.seed, 10, dt=dt))
    batch = sdm.Batch(runs, use_graph=use_graph, graph_steps=4)
    batch.step(3).step(7)
    torch.cuda.synchronize()
    for r, a in zip(runs, alone):
        x1, v1 = r.attributes()
        x2, v2 = a.attributes()
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
        assert r.info().step == 10
    batch.close()


def test_invalid_attributes_rejected(env):
    O, sdm, torch = env
    run = sdm.Run(sdm.make_config("golovin", n_cells=2), 8)
    xi = np.ones(4, np.int64)
    v = np.full(4, 1e-15)
    with pytest.raises(sdm.SdmError) as e:
        run.set_attributes(xi, np.array([1e-15, -1.0, 1e-15, 1e-15]), np.zeros(4, np.int32))
    assert e.value.status == sdm.SDM_EINVAL and "SD 1" in str(e.value)
    with pytest.raises(sdm.SdmError):
        run.set_attributes(xi, v, np.array([0, 1, 2, 0], np.int32))
    with pytest.raises(sdm.SdmError):
        run.set_attributes(np.array([1, -3, 1, 1], np.int64), v, np.zeros(4, np.int32))
    with pytest.raises(sdm.SdmError) as e:
        run.step(1)
    assert e.value.status == sdm.SDM_ESTATE
    run.set_attributes(xi, v, np.array([0, 1, 1, 0], np.int32)).step(2)
    run.close()
