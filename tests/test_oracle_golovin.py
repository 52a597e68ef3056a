"""Pins of the oracle against the Golovin closed form (the paper's Box example
compares its Golovin run with the analytic solution of the Smoluchowski
equation): first the closed form itself, then the SDM ensemble."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import golovin as G
from paper_2103_17238_gb300 import inputs as I

B = I.GOLOVIN_B
N0 = I.N_CONC_BOX
X0 = I.x0_box()


@pytest.mark.parametrize("t", [0.0, 600.0, 1200.0, 3600.0])
def test_closed_form_moments(t):
    """zeroth moment N0 (1 - tau) = N0 exp(-b N0 x0 t); first moment N0 x0 (volume conserved)."""
    # integrate over u = x / x0 on geometric pieces
    f0 = lambda u: G.number_density(u * X0, t, b=B, n0=N0, x0=X0) * X0
    f1 = lambda u: u * X0 * G.number_density(u * X0, t, b=B, n0=N0, x0=X0) * X0
    cuts = np.concatenate([[0.0], np.geomspace(1e-6, 1e7, 80)])
    m0 = sum(integrate.quad(f0, a, b, limit=200, epsrel=1e-12, epsabs=0)[0] for a, b in zip(cuts[:-1], cuts[1:]))
    m1 = sum(integrate.quad(f1, a, b, limit=200, epsrel=1e-12, epsabs=0)[0] for a, b in zip(cuts[:-1], cuts[1:]))
    assert m0 == pytest.approx(G.total_number(t, b=B, n0=N0, x0=X0), rel=1e-10)
    assert m1 == pytest.approx(N0 * X0, rel=1e-10)


def test_closed_form_small_time_limit():
    x = X0 * np.array([0.1, 1.0, 3.0])
    assert np.allclose(G.number_density(x, 1e-6, b=B, n0=N0, x0=X0),
                       G.number_density(x, 0.0, b=B, n0=N0, x0=X0), rtol=1e-6)


def test_initial_sample_matches_exponential_spectrum(oracle_lib):
    O = oracle_lib
    inst = I.box_golovin(2**12)
    st = O.State(inst.xi.copy(), inst.v.copy(), inst.cell, None, 1)
    P = O.params("golovin", dv=inst.dv)
    got = O.spectrum(P, st, I.R_EDGES)
    want = G.dv_dlnr_bins(I.R_EDGES, 0.0, b=B, n0=N0, x0=X0)
    big = want > 1e-2 * want.max()
    assert np.allclose(got[big], want[big], rtol=0.05)
    # the product integrates back to the total volume in range
    vol = np.sum(got * np.diff(np.log(I.R_EDGES))) * inst.dv
    r = np.array([O.radius(t) for t in inst.v])
    inside = (r >= I.R_EDGES[0]) & (r < I.R_EDGES[-1])
    assert vol == pytest.approx(math.fsum(inst.xi[inside] * inst.v[inside]), rel=1e-12)


def _ensemble(n_sd, seeds, t_out):
    from oracle import oracle as O

    P = O.params("golovin", dv=I.DV_BOX)
    nums = {t: [] for t in t_out}
    specs = {t: [] for t in t_out}
    for seed in seeds:
        inst = I.box_golovin(n_sd)
        st = O.State(inst.xi.copy(), inst.v.copy(), inst.cell, None, 1)
        P.seed = seed
        done = 0
        for t in t_out:
            O.run(P, st, done, t - done)
            done = t
            nums[t].append(st.xi.sum() / I.DV_BOX)
            specs[t].append(O.spectrum(P, st, I.R_EDGES))
    return nums, specs


def test_ensemble_number_decay_and_spectrum():
    """SDM ensemble mean vs the closed form at t = 1200, 2400, 3600 s.

    Total number: within 3 standard errors plus a finite-n_sd bias allowance
    of 4 %.  A wrong scale factor (e.g. dropping [n_c(n_c-1)/2]/floor(n_c/2)
    or doubling it) moves N(3600) by orders of magnitude.  Spectrum: relative
    L1 error over bins holding >= 1e-3 of the peak must be below 0.25 at
    n_sd = 2^12 and shrink at n_sd = 2^14."""
    t_out = [1200, 2400, 3600]
    errs = {}
    for n_sd, seeds in [(2**12, range(4)), (2**14, range(2))]:
        nums, specs = _ensemble(n_sd, seeds, t_out)
        for t in t_out:
            want_n = G.total_number(t, b=B, n0=N0, x0=X0)
            got = np.array(nums[t])
            se = got.std(ddof=1) / math.sqrt(len(got)) if len(got) > 1 else 0.0
            assert abs(got.mean() - want_n) <= 3 * se + 0.04 * want_n, (n_sd, t)
            want = G.dv_dlnr_bins(I.R_EDGES, t, b=B, n0=N0, x0=X0)
            mask = want >= 1e-3 * want.max()
            mean = np.mean(specs[t], axis=0)
            errs[(n_sd, t)] = np.abs(mean[mask] - want[mask]).sum() / want[mask].sum()
    for t in t_out:
        assert errs[(2**12, t)] < 0.25, errs
    assert sum(errs[(2**14, t)] for t in t_out) < sum(errs[(2**12, t)] for t in t_out), errs
