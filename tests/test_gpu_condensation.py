"""Parity of the condensation step (sdm_condensation_step) with the oracle.

Volumes must match bit for bit (the binary32 change of volume and the
binary64 add are reproduced operation by operation); the per-cell condensed
water sums in another order than the oracle, so it is compared within the
summation bound 2 n u sum |xi dV| (u = 2^-53, n summands per cell)."""
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


def _check_condensed(got, want, st_xi, st_cell, dv_abs):
    n_cells = len(want)
    for c in range(n_cells):
        m = (st_cell == c) & (st_xi > 0)
        bound = 2 * max(1, int(m.sum())) * U * float(np.sum(np.abs(st_xi[m].astype(np.float64) * dv_abs[m]))) + 1e-300
        assert abs(got[c] - want[c]) <= bound, (c, got[c], want[c], bound)


def _ragged(rng, sizes):
    cell = np.concatenate([np.full(n, c, np.int32) for c, n in enumerate(sizes)])
    n = len(cell)
    xi = rng.integers(1, 10**9, n).astype(np.int64)
    xi[rng.random(n) < 0.05] = 0
    r = np.exp(rng.uniform(np.log(5e-7), np.log(2e-3), n))
    v = 4 / 3 * np.pi * r**3
    cell[rng.random(n) < 0.02] = -1  # outside the domain
    perm = rng.permutation(n)
    return xi[perm], v[perm], cell[perm]


SIZES = [0, 1, 2, 3, 64, 255, 256, 257, 511, 513, 1000, 4097, 20001]


@pytest.mark.parametrize("kernel", ["geometric", "golovin"])
def test_condensation_with_coalescence_ragged(env, kernel):
    """Ragged cells (empty, odd, work items split at 256 slots, a 20001-SD
    cell), dead SDs and SDs outside the domain; per-cell G and s with growth,
    evaporation down to the floor and s = 0; condensation and coalescence
    interleaved for 4 steps, state and condensed water against the oracle."""
    O, sdm, torch = env
    rng = np.random.default_rng(23)
    xi, v, cell = _ragged(rng, SIZES)
    nc = len(SIZES)
    G = rng.uniform(0.5e-10, 1.5e-10, nc)
    s = rng.choice([0.01, -0.05, 0.0, 0.002, -0.9], nc)
    dv_cell = 1e3 if kernel == "geometric" else 1e-2
    r_min = 1e-6
    run = sdm.Run(sdm.make_config(kernel, dv=dv_cell, dt=2.0, n_cells=nc, seed=3), len(xi))
    run.set_attributes(xi, v, cell)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nc)
    P = O.params(kernel, dv=dv_cell, dt=2.0, seed=3)
    for step in range(4):
        v_before = st.v.copy()
        want = O.condense(P, st, G, s, r_min)
        got = run.condense(G, s, r_min)
        _check_condensed(got, want, st.xi, st.cell, np.abs(st.v - v_before))
        O.step(P, st, step)
        run.step(1)
    gx, gv = run.attributes()
    assert np.array_equal(gx, st.xi)
    assert np.array_equal(gv, st.v)
    assert int((gv != v).sum()) > len(v) // 2
    run.close()


def test_condensation_full_grid(env):
    """The benchmark grid (4.19M SDs), a supersaturation field varying over
    the cells (growth in half of them, evaporation in the other), 6 cycles
    of condensation then coalescence, every SD against the oracle."""
    O, sdm, torch = env
    g = I.grid_geometric(seed=2)
    rng = np.random.default_rng(5)
    G = np.full(g.n_cells, 1.1e-10)
    s = rng.uniform(-0.02, 0.02, g.n_cells)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=2), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell)
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, g.n_cells)
    P = O.params("geometric", dv=g.dv, seed=2)
    for step in range(6):
        want = O.condense(P, st, G, s, 1e-6, want_condensed=(step == 5))
        got = run.condense(G, s, 1e-6, want_condensed=(step == 5))
        O.step(P, st, step)
        run.step(1)
    gx, gv = run.attributes()
    assert np.array_equal(gx, st.xi)
    assert np.array_equal(gv, st.v)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-30)
    run.close()


def test_condensed_water_to_device_and_zero_supersaturation(env):
    O, sdm, torch = env
    g = I.grid_geometric(side=4, sd_per_cell=256, seed=4)
    run = sdm.Run(sdm.make_config("geometric", dv=g.dv, n_cells=g.n_cells, seed=4), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell)
    G = np.full(g.n_cells, 1e-10)
    out = torch.empty(g.n_cells, dtype=torch.float64, device="cuda")
    sdm.sdm_condensation_step(run.h, G, np.zeros(g.n_cells), 1e-6, out=out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    gx, gv = run.attributes()
    assert np.array_equal(gv, g.v)  # s = 0: no SD changes
    s = np.full(g.n_cells, 0.01)
    sdm.sdm_condensation_step(run.h, G, s, 1e-6, out=out)
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, g.n_cells)
    want = O.condense(O.params("geometric", dv=g.dv), st, G, s, 1e-6)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)
    run.close()


def test_condensation_rejects_bad_inputs(env):
    O, sdm, torch = env
    run = sdm.Run(sdm.make_config("geometric", n_cells=2), 8)
    with pytest.raises(sdm.SdmError) as e:
        run.condense([1e-10, 1e-10], [0.0, 0.0], 1e-6)
    assert e.value.status == sdm.SDM_ESTATE
    run.set_attributes(np.ones(4, np.int64), np.full(4, 1e-15), np.array([0, 1, 1, 0], np.int32))
    for G, s, rmin in (([-1e-10, 1e-10], [0.0, 0.0], 1e-6), ([1e-10, 1e-10], [0.0, 1.5], 1e-6),
                       ([1e-10, 1e-10], [0.0, 0.0], 0.0), ([1e-10, 1e-2], [0.0, 0.5], 1e-6),
                       ([1e-10, np.nan], [0.0, 0.0], 1e-6)):
        with pytest.raises(sdm.SdmError) as e:
            run.condense(G, s, rmin)
        assert e.value.status == sdm.SDM_EINVAL
    run.condense([1e-10, 1e-10], [0.01, -0.01], 1e-6)
    run.close()
