"""Pins of the oracle's dv/dlnr product in its per-cell form (paper: API in
brief, the ParticlesVolumeSpectrum product): a hand-worked two-cell case
with dyadic volumes, the volume that each cell's spectrum integrates back
to, and the relation between the per-cell and the total forms."""
import math

import numpy as np
import pytest

# radius bins [1, 10), [10, 100), [100, 1000) um: Delta ln r = ln 10 each
EDGES = np.array([1e-6, 1e-5, 1e-4, 1e-3])
# dyadic volumes and the bins of their radii (3 v / 4 pi)^(1/3):
# 2^-50 m^3 -> 5.97 um, 2^-40 m^3 -> 59.7 um, 2^-30 m^3 -> 597 um
V0, V1, V2 = 2.0**-50, 2.0**-40, 2.0**-30


def _two_cells(O):
    xi = np.array([4, 2, 8, 1, 0, 5, 3], np.int64)
    v = np.array([V0, V1, V0, V2, V1, V1, V2])
    cell = np.array([0, 0, 1, 1, 1, -1, 0], np.int32)  # SD 4 dead, SD 5 outside the domain
    return O.State(xi, v, cell, None, 2)


def test_per_cell_hand_case(oracle_lib):
    """Per cell, bin b: sum(xi v) of its live SDs in the bin / dV / Delta ln r."""
    O = oracle_lib
    for r, b in ((O.radius(V0), 0), (O.radius(V1), 1), (O.radius(V2), 2)):
        assert EDGES[b] <= r < EDGES[b + 1]
    dv = 2.0
    P = O.params("golovin", dv=dv)
    got = O.spectrum(P, _two_cells(O), EDGES, per_cell=True)
    ln10 = math.log(10.0)
    want = np.array([[4 * V0, 2 * V1, 3 * V2],
                     [8 * V0, 0.0, 1 * V2]]) / dv / ln10
    assert got.shape == (2, 3)
    assert np.allclose(got, want, rtol=1e-15, atol=0.0)


def test_per_cell_integrates_to_the_cells_water(oracle_lib):
    """sum_b dv/dlnr(c, b) Delta ln r_b dV is the water volume of cell c
    (all of its live SDs inside the edges), computed here from the state
    without any binning."""
    O = oracle_lib
    rng = np.random.default_rng(21)
    n_cells, n = 5, 400
    xi = rng.integers(0, 1000, n).astype(np.int64)
    v = np.exp(rng.uniform(np.log(1e-17), np.log(1e-10), n))
    cell = rng.integers(-1, n_cells, n).astype(np.int32)
    st = O.State(xi, v, cell, None, n_cells)
    dv = 1e3
    P = O.params("geometric", dv=dv)
    got = O.spectrum(P, st, EDGES, per_cell=True)
    dln = np.diff(np.log(EDGES))
    r = np.cbrt(3.0 * v / (4.0 * math.pi))
    inside = (r >= EDGES[0]) & (r < EDGES[-1]) & (xi > 0)
    for c in range(n_cells):
        m = inside & (cell == c)
        water = math.fsum(xi[m] * v[m])
        assert np.sum(got[c] * dln) * dv == pytest.approx(water, rel=1e-13)


def test_total_is_the_cell_mean_of_the_per_cell_spectra(oracle_lib):
    """The total form divides by dV n_cells: per-cell values times dV,
    summed over cells, equal the total times dV n_cells."""
    O = oracle_lib
    st = _two_cells(O)
    P = O.params("golovin", dv=2.0)
    per = O.spectrum(P, st, EDGES, per_cell=True)
    tot = O.spectrum(P, st, EDGES, per_cell=False)
    assert np.allclose(per.sum(axis=0) * 2.0, tot * 2.0 * 2, rtol=1e-15, atol=0.0)
    assert np.allclose(tot, per.mean(axis=0), rtol=1e-15, atol=0.0)
