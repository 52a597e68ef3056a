"""Seeded synthetic inputs for the SDM coalescence workloads.

This module holds no arithmetic of the coalescence step itself; it only
produces initial super-droplet attributes (multiplicity xi, volume v, cell)
and run descriptions.  Both the CUDA path's tests/benchmarks and the oracle's
tests draw their inputs from here.

Initialisation follows the paper's worked example (API in brief): an initial
spectrum sampled "deterministically" so that every super-droplet starts with
the same multiplicity.  The sampling points are the mid-quantiles
q_i = (i + 1/2) / n_sd of the number distribution, so that each SD stands for
1/n_sd of the droplets: xi_i = round(N / n_sd), with N the droplet count of
the cell.

Workloads (all SI units):
  box_golovin       one cell, dV = 1e6 m^3, exponential spectrum with mean
                    radius 30.531 um (x0 = 4/3 pi r^3 = 1.1921e-13 m^3) and
                    2^23 m^-3 droplets, Golovin b = 1500 s^-1, dt = 1 s;
                    n_sd = 2^12 (small case) or 2^20 (large single cell).
  grid_geometric    128 x 128 cells of dV = 1e3 m^3, 256 SDs per cell,
                    lognormal spectrum (geometric-mean radius 15 um,
                    sigma_g = 1.4, 1e8 m^-3), geometric kernel, dt = 1 s.
  batched_ensemble  1024 Golovin box instances, n_sd = round(2^U(8,16)) drawn
                    with numpy default_rng(3), instance seeds 0..1023.
  serving_stream    Poisson arrivals (200 /s, default_rng(4)) of Golovin boxes
                    or geometric grids with n_sd = round(2^U(10,20)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import special

MEAN_RADIUS_BOX = 30.531e-6  # m
N_CONC_BOX = 2.0**23  # m^-3
DV_BOX = 1.0e6  # m^3
GOLOVIN_B = 1500.0  # s^-1

GRID_SIDE = 128
SD_PER_CELL_GRID = 256
DV_GRID = 1.0e3  # m^3
LOGNORMAL_RADIUS = 15.0e-6  # m
LOGNORMAL_SIGMA = 1.4
N_CONC_GRID = 1.0e8  # m^-3

# radius bin edges of the paper's spectrum product: 32 log-spaced edges, 10 um .. 5 mm
R_EDGES = np.logspace(np.log10(10.0e-6), np.log10(5.0e3 * 1e-6), num=32)


def sphere_volume(r):
    return 4.0 / 3.0 * np.pi * np.asarray(r, dtype=np.float64) ** 3


def x0_box() -> float:
    return float(sphere_volume(MEAN_RADIUS_BOX))


def _quantiles(n_sd: int) -> np.ndarray:
    return (np.arange(n_sd, dtype=np.float64) + 0.5) / n_sd


def exponential_sample(n_sd: int, n_total: float, x0: float):
    """Constant-multiplicity sample of n(x) = N/x0 exp(-x/x0): volumes at the
    mid-quantiles, equal multiplicities round(N / n_sd)."""
    q = _quantiles(n_sd)
    v = -x0 * np.log1p(-q)
    xi = np.full(n_sd, int(round(n_total / n_sd)), dtype=np.int64)
    return xi, v


def lognormal_sample(n_sd: int, n_total: float, r_g: float, sigma_g: float):
    """Constant-multiplicity sample of a lognormal radius distribution."""
    q = _quantiles(n_sd)
    r = r_g * np.exp(np.log(sigma_g) * special.ndtri(q))
    xi = np.full(n_sd, int(round(n_total / n_sd)), dtype=np.int64)
    return xi, sphere_volume(r)


@dataclass
class Instance:
    """One independent coalescence run (a box or a grid of cells)."""

    kernel: str  # "golovin" | "geometric"
    xi: np.ndarray
    v: np.ndarray
    cell: np.ndarray  # int32, cell-major order
    n_cells: int
    dv: float
    dt: float
    seed: int
    steps: int = 0
    b: float = GOLOVIN_B
    meta: dict = field(default_factory=dict)

    @property
    def n_sd(self) -> int:
        return int(self.xi.shape[0])


def box_golovin(n_sd: int = 2**12, seed: int = 0, steps: int = 3600) -> Instance:
    xi, v = exponential_sample(n_sd, N_CONC_BOX * DV_BOX, x0_box())
    return Instance("golovin", xi, v, np.zeros(n_sd, np.int32), 1, DV_BOX, 1.0, seed, steps)


def grid_geometric(side: int = GRID_SIDE, sd_per_cell: int = SD_PER_CELL_GRID, seed: int = 0,
                   steps: int = 600) -> Instance:
    """Every cell holds the same mid-quantile lognormal sample; cells diverge
    through their random streams."""
    xi1, v1 = lognormal_sample(sd_per_cell, N_CONC_GRID * DV_GRID, LOGNORMAL_RADIUS, LOGNORMAL_SIGMA)
    n_cells = side * side
    xi = np.tile(xi1, n_cells)
    v = np.tile(v1, n_cells)
    cell = np.repeat(np.arange(n_cells, dtype=np.int32), sd_per_cell)
    return Instance("geometric", xi, v, cell, n_cells, DV_GRID, 1.0, seed, steps)


def batched_ensemble(n_inst: int = 1024, lo_log2: float = 8.0, hi_log2: float = 16.0,
                     rng_seed: int = 3, steps: int = 1800) -> list[Instance]:
    rng = np.random.default_rng(rng_seed)
    sizes = np.round(2.0 ** rng.uniform(lo_log2, hi_log2, size=n_inst)).astype(np.int64)
    out = []
    for i, n in enumerate(sizes):
        out.append(box_golovin(int(n), seed=i, steps=steps))
    return out


@dataclass
class Request:
    arrival: float  # s since stream start
    inst: Instance


def serving_stream(n_requests: int = 2000, rate: float = 200.0, rng_seed: int = 4,
                   lo_log2: float = 10.0, hi_log2: float = 20.0) -> list[Request]:
    """Poisson arrivals of box or grid runs with random size, length, dt and spectrum."""
    rng = np.random.default_rng(rng_seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        kind = "golovin" if rng.random() < 0.5 else "geometric"
        n_sd = int(round(2.0 ** rng.uniform(lo_log2, hi_log2)))
        steps = int(rng.integers(100, 1001))
        dt = float(rng.choice([0.5, 1.0, 2.0]))
        spec = "exponential" if rng.random() < 0.5 else "lognormal"
        if kind == "golovin":
            n_cells, dv, per = 1, DV_BOX, n_sd
        else:
            per = SD_PER_CELL_GRID
            n_cells = max(1, n_sd // per)
            per = n_sd // n_cells
            dv = DV_GRID
        if spec == "exponential":
            xi1, v1 = exponential_sample(per, N_CONC_BOX * dv, x0_box())
        else:
            xi1, v1 = lognormal_sample(per, N_CONC_GRID * dv, LOGNORMAL_RADIUS, LOGNORMAL_SIGMA)
        inst = Instance(kind, np.tile(xi1, n_cells), np.tile(v1, n_cells),
                        np.repeat(np.arange(n_cells, dtype=np.int32), per), n_cells, dv, dt,
                        seed=1000 + i, steps=steps, meta={"spectrum": spec})
        out.append(Request(t, inst))
    return out
