"""Pins of the oracle's sedimentation step: hand-worked falls, the fall
distance against the Rogers-Yau formula evaluated independently, whole
trajectories against exact rational arithmetic, conservation of water
(inside plus precipitated), and SDs outside the domain left alone by the
coalescence step and the spectrum."""
import math
from fractions import Fraction

import numpy as np
import pytest


def test_fall_hand_cases(oracle_lib):
    O = oracle_lib
    assert O.fall(5.0, 3, 1.5, 8.0) == (3, 3.5)          # stays in its level
    assert O.fall(1.0, 3, 3.0, 8.0) == (2, 6.0)          # one level down
    assert O.fall(1.0, 3, 17.5, 8.0) == (0, 7.5)         # three levels at once
    assert O.fall(1.0, 0, 2.0, 8.0) == (-1, 0.0)         # through the bottom
    assert O.fall(1.0, 2, 17.5, 8.0) == (-1, 0.0)
    assert O.fall(1.0, 2, 17.0, 8.0) == (0, 0.0)         # exactly at the domain bottom: still inside
    assert O.fall(3.0, 2, 3.0, 8.0) == (2, 0.0)          # lands on its level's bottom: stays
    assert O.fall(0.0, 2, 8.0, 8.0) == (1, 0.0)          # a whole level
    # zeta - d = -2^-60; -2^-60 + 10 rounds to 10: the SD is on the boundary
    # and stays in the level above at zeta 0
    assert O.fall(2.0**-60, 3, 2.0**-59, 10.0) == (3, 0.0)
    assert O.fall(0.5, 4, 0.0, 8.0) == (4, 0.5)          # no fall


@pytest.mark.parametrize("r_um", [2.0, 15.0, 35.0, 80.0, 300.0, 900.0, 2500.0])
def test_fall_distance_is_the_rogers_yau_speed_times_dt(oracle_lib, r_um):
    """v_t(r) dt for r in each regime: k1 r^2 below 40 um, k2 r to 600 um,
    k3 sqrt(r) above, evaluated here in binary64 from the radius of the
    volume, within the binary32 rounding of the oracle's evaluation."""
    O = oracle_lib
    for dt in (1.0, 0.25, 7.0):
        P = O.params("geometric", dt=dt)
        r = r_um * 1e-6
        v = 4.0 / 3.0 * math.pi * r**3
        rr = (v * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        if rr < 40e-6:
            want = 1.19e8 * rr * rr
        elif rr < 600e-6:
            want = 8.0e3 * rr
        else:
            want = 201.0 * math.sqrt(rr)
        got = O.fall_distance(P, v)
        assert got == float(np.float32(got))                  # a binary32 value
        assert abs(got - want * dt) <= 4e-7 * want * dt, (r_um, dt, got, want * dt)


def _exact_trajectory(z0, d, dz, nx, cell0, steps):
    """(cell, zeta) after each step in exact rational arithmetic; cell -1
    once the SD has left through the bottom."""
    iz, ix = divmod(cell0, nx)
    z = Fraction(iz) * Fraction(dz) + Fraction(z0)
    out = []
    for _ in range(steps):
        z -= Fraction(d)
        if z < 0:
            out.append((-1, 0.0))
            break
        lvl = math.floor(z / Fraction(dz))
        out.append((lvl * nx + ix, float(z - lvl * Fraction(dz))))
    return out


def test_trajectories_are_exact_for_dyadic_heights(oracle_lib):
    """With dz = 8 and heights on a 2^-10 grid, every subtraction and level
    change of the fall is exact in binary64: the oracle must land every SD in
    the cell and at the height that exact arithmetic gives, step by step,
    including the steps at which SDs leave through the bottom."""
    O = oracle_lib
    rng = np.random.default_rng(11)
    nx, nz, dz = 3, 5, 8.0
    n = 300
    r = np.exp(rng.uniform(np.log(5e-6), np.log(3e-3), n))
    v = 4.0 / 3.0 * np.pi * r**3
    xi = rng.integers(1, 10**6, n).astype(np.int64)
    cell = rng.integers(0, nx * nz, n).astype(np.int32)
    zeta = np.floor(rng.uniform(0, dz, n) * 1024.0) / 1024.0
    P = O.params("geometric", dt=3.0)
    d = np.array([O.fall_distance(P, x) for x in v])
    want = [_exact_trajectory(zeta[i], d[i], dz, nx, int(cell[i]), 40) for i in range(n)]
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nx * nz)
    zt = zeta.copy()
    precip_total = 0.0
    for t in range(40):
        precip_total += O.sediment(P, st, nx, dz, zt)
        for i in range(n):
            w = want[i][t] if t < len(want[i]) else (-1, 0.0)
            assert (int(st.cell[i]), float(zt[i])) == w, (i, t)
    left = st.cell < 0
    assert 0 < left.sum() < n
    assert math.isclose(precip_total, float(np.sum(xi[left] * v[left])), rel_tol=1e-13)


def test_water_is_conserved_and_outside_sds_are_left_alone(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(5)
    nx, nz, dz = 4, 6, 10.0
    n = 2000
    r = np.exp(rng.uniform(np.log(3e-6), np.log(4e-3), n))
    v = 4.0 / 3.0 * np.pi * r**3
    xi = rng.integers(1, 10**9, n).astype(np.int64)
    xi[rng.random(n) < 0.05] = 0
    cell = rng.integers(0, nx * nz, n).astype(np.int32)
    zeta = rng.uniform(0, dz, n)
    P = O.params("geometric", dt=5.0, dv=1e3)
    st = O.State(xi.copy(), v.copy(), cell.copy(), None, nx * nz)
    total0 = math.fsum(xi * v)
    precip = 0.0
    for s in range(30):
        pre = (st.xi.copy(), st.v.copy())
        precip += O.sediment(P, st, nx, dz, zeta)
        inside = st.cell >= 0
        assert np.array_equal(st.xi, pre[0]) and np.array_equal(st.v, pre[1])  # sedimentation changes no xi, v
        assert np.all(zeta[inside] >= 0) and np.all(zeta[inside] < dz)
        assert np.all(st.cell[xi == 0] == -1)                        # dead SDs left at the first step
        assert np.all(st.cell[inside] % nx == cell[inside] % nx)     # columns are kept
        assert np.all(st.cell[inside] // nx <= cell[inside] // nx)   # only downwards
        assert math.isclose(math.fsum(st.xi[inside] * st.v[inside]) + precip, total0, rel_tol=1e-12)
        # coalescence ignores SDs outside; the spectrum does not count them
        before = (st.xi.copy(), st.v.copy())
        O.step(P, st, s)
        assert np.array_equal(st.xi[~inside], before[0][~inside])
        assert np.array_equal(st.v[~inside], before[1][~inside])
    edges = np.logspace(np.log10(1e-6), np.log10(1e-2), 20)
    full = O.spectrum(P, st, edges)
    only_in = O.State(st.xi.copy(), st.v.copy(), st.cell.copy(), None, nx * nz)
    only_in.xi[st.cell < 0] = 0
    assert np.array_equal(full, O.spectrum(P, only_in, edges))
    assert (st.cell < 0).sum() > (xi == 0).sum()                     # some fell through the bottom


def test_height_conversions(oracle_lib):
    O = oracle_lib
    z = np.array([0.0, 7.5, 8.0, 39.999, 12.25])
    cell = np.array([0 * 3 + 1, 0 * 3 + 2, 1 * 3 + 0, 4 * 3 + 1, 1 * 3 + 2], dtype=np.int32)
    zeta = O.zeta_of(z, cell, 3, 8.0)
    assert np.allclose(zeta, [0.0, 7.5, 0.0, 39.999 - 32.0, 4.25], rtol=0, atol=1e-15)
    assert np.array_equal(O.z_of(zeta, cell, 3, 8.0), z)
