"""Closed-form solution of the Smoluchowski equation for the Golovin kernel.

TEST INFRASTRUCTURE ONLY (see ``oracle.py``).  The paper's Box example with the
Golovin additive kernel K = b (x + y) is compared against "the analytical
solution of the Smoluchowski equation" (paper: Usage examples, Box environment
examples).  This module restates that solution from the mathematics (Golovin
1963): for an initially exponential number density over droplet volume x,

    n(x, 0) = N0 / x0 * exp(-x / x0),

the mean-field solution is

    n(x, t) = N0 (1 - tau) / (x sqrt(tau)) * exp(-(1 + tau) x / x0)
              * I1(2 x sqrt(tau) / x0),
    tau     = 1 - exp(-b N0 x0 t),

with N0 the number concentration, x0 the mean volume, I1 the modified Bessel
function.  The total number decays as N(t) = N0 exp(-b N0 x0 t); the volume
concentration N0 x0 is conserved.  The mass density per unit ln r is
dv/dlnr = 3 x^2 n(x).  I1 is evaluated through scipy's exponentially scaled
``ive`` so that the exponentials combine to exp(-(1 - sqrt(tau))^2 x / x0).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, special


def tau(b, n0, x0, t):
    return -np.expm1(-b * n0 * x0 * t)


def number_density(x, t, *, b, n0, x0):
    """n(x, t): droplets per m^3 of air per m^3 of droplet volume."""
    x = np.asarray(x, dtype=np.float64)
    if t == 0:
        return n0 / x0 * np.exp(-x / x0)
    T = tau(b, n0, x0, t)
    sq = np.sqrt(T)
    z = 2.0 * x * sq / x0
    return n0 * (1.0 - T) / (x * sq) * np.exp(-((1.0 - sq) ** 2) * x / x0) * special.ive(1, z)


def total_number(t, *, b, n0, x0):
    return n0 * np.exp(-b * n0 * x0 * t)


def dv_dlnr_bins(r_edges, t, *, b, n0, x0):
    """Bin averages of dv/dlnr over [r_e, r_{e+1}):  (integral of x n(x) dx) / d ln r."""
    r_edges = np.asarray(r_edges, dtype=np.float64)
    out = np.zeros(len(r_edges) - 1)
    for i in range(len(out)):
        xa = 4.0 / 3.0 * np.pi * r_edges[i] ** 3
        xb = 4.0 / 3.0 * np.pi * r_edges[i + 1] ** 3
        # integrate in ln x for accuracy across decades
        f = lambda lx: np.exp(lx) * np.exp(lx) * number_density(np.exp(lx), t, b=b, n0=n0, x0=x0)
        val, _ = integrate.quad(f, np.log(xa), np.log(xb), limit=200, epsabs=0.0, epsrel=1e-10)
        out[i] = val / (np.log(r_edges[i + 1]) - np.log(r_edges[i]))
    return out
