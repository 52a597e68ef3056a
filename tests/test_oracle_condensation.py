"""Pins of the oracle's condensation step: the large-drop limit of the
diffusional growth law, r dr/dt = s G, makes r^2 grow linearly in time
(exactly, for constant s and G); the floor radius stops evaporation; the
condensed water per cell is the change of sum(xi v); SDs that are dead or
outside the domain are left alone."""
import math

import numpy as np
import pytest


def _state(O, r, xi=None, cell=None, n_cells=1):
    r = np.asarray(r, np.float64)
    v = 4.0 / 3.0 * math.pi * r**3
    xi = np.ones(len(r), np.int64) if xi is None else np.asarray(xi, np.int64)
    cell = np.zeros(len(r), np.int32) if cell is None else np.asarray(cell, np.int32)
    return O.State(xi, v, cell, None, n_cells)


def _radius(v):
    return np.cbrt(3.0 * np.asarray(v) / (4.0 * math.pi))


def test_zero_supersaturation_leaves_volumes_bitwise(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(1)
    st = _state(O, np.exp(rng.uniform(np.log(1e-6), np.log(2e-3), 500)))
    v0 = st.v.copy()
    out = O.condense(O.params(dt=1.0), st, [1e-10], [0.0], 1e-6)
    assert np.array_equal(st.v, v0) and out[0] == 0.0


@pytest.mark.parametrize("s", [0.003, -0.002])
def test_r_squared_grows_linearly(oracle_lib, s):
    """After n steps of dt with constant G and s, r^2 = r0^2 + 2 G s n dt
    (closed form of the growth law's large-drop limit), to the binary32
    rounding of each step's change (relative 1e-6 of the change per step)."""
    O = oracle_lib
    G, dt, n = 1.2e-10, 2.0, 50
    r0 = np.array([8e-6, 15e-6, 40e-6, 300e-6])
    st = _state(O, r0)
    P = O.params(dt=dt)
    for _ in range(n):
        O.condense(P, st, [G], [s], 1e-7)
    want_x = r0**2 + 2.0 * G * s * n * dt
    got_x = _radius(st.v) ** 2
    change = np.abs(want_x - r0**2)
    assert np.all(np.abs(got_x - want_x) <= 2e-6 * change * n ** 0.5 + 2e-6 * want_x * 2.0**-23 * n)
    assert np.all(np.abs(got_x - want_x) / want_x < 1e-6)


def test_hand_worked_step(oracle_lib):
    """r0 = 10 um, G = 1e-10 m^2/s, s = 0.01, dt = 1 s: r1^2 = 1.02e-10 m^2,
    dV = 4/3 pi (r1^3 - r0^3) = 4/3 pi (1.02^1.5 - 1) 1e-15 m^3."""
    O = oracle_lib
    st = _state(O, [10e-6], xi=[7])
    out = O.condense(O.params(dt=1.0), st, [1e-10], [0.01], 1e-6)
    dv = 4.0 / 3.0 * math.pi * (1.02**1.5 - 1.0) * 1e-15
    assert st.v[0] == pytest.approx(4.0 / 3.0 * math.pi * 1e-15 + dv, rel=1e-6)
    assert out[0] == pytest.approx(7 * dv, rel=1e-5)


def test_evaporation_stops_at_the_floor(oracle_lib):
    """Strong subsaturation: radii above r_min end at r_min; radii already
    below r_min do not change."""
    O = oracle_lib
    r_min = 2e-6
    st = _state(O, [1e-6, 2.5e-6, 5e-6, 50e-6])
    v0 = st.v.copy()
    O.condense(O.params(dt=10.0), st, [1e-10], [-0.5], r_min)
    r = _radius(st.v)
    assert st.v[0] == v0[0]
    assert np.allclose(r[1:3], r_min, rtol=1e-6)
    assert r[3] < 50e-6 and r[3] > r_min
    assert np.sqrt(50e-6**2 - 2 * 1e-10 * 0.5 * 10.0) == pytest.approx(r[3], rel=1e-6)


def test_condensed_water_per_cell(oracle_lib):
    """condensed[c] = change of sum(xi v) over cell c (different s per cell,
    growth and evaporation); dead SDs and SDs outside the domain keep their
    volume and add nothing."""
    O = oracle_lib
    rng = np.random.default_rng(4)
    n, nc = 600, 5
    r = np.exp(rng.uniform(np.log(2e-6), np.log(1e-3), n))
    xi = rng.integers(0, 10**6, n).astype(np.int64)
    cell = rng.integers(-1, nc, n).astype(np.int32)
    st = _state(O, r, xi, cell, nc)
    v0 = st.v.copy()
    G = rng.uniform(0.5e-10, 1.5e-10, nc)
    s = np.array([0.01, -0.01, 0.0, 0.002, -0.3])
    out = O.condense(O.params(dt=1.0), st, G, s, 1e-6)
    idle = (xi == 0) | (cell < 0)
    assert np.array_equal(st.v[idle], v0[idle])
    for c in range(nc):
        m = (cell == c) & (xi > 0)
        want = math.fsum(xi[m] * (st.v[m] - v0[m]))
        assert out[c] == pytest.approx(want, rel=1e-9, abs=1e-30)
    assert out[2] == 0.0
    assert out[0] > 0 and out[1] < 0


def test_rejects_a_non_positive_floor(oracle_lib):
    O = oracle_lib
    st = _state(O, [1e-5])
    with pytest.raises(ValueError):
        O.condense(O.params(), st, [1e-10], [0.0], 0.0)
