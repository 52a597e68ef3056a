"""Pins of the oracle's per-pair arithmetic: hand-worked Shima updates with
dyadic volumes (exact), the collision count gamma = ceil(p - u) and its cap,
the probability scale factor, the cube root against libm, and the Rogers-Yau
terminal velocity against measured fall speeds."""
import math

import numpy as np
import pytest


# (xi_j, xi_k, gamma) -> (xi_j', xi_k', v_j', v_k') with v_j = 0.25, v_k = 0.5,
# worked by hand from the Shima rules: unequal -> xi_j -= gamma xi_k and
# v_k += gamma v_j; xi_j - gamma xi_k == 0 -> split the k SD in halves, both
# with volume v_k + gamma v_j.
HAND = [
    ((10, 3, 2), (4, 3, 0.25, 1.0)),
    ((6, 3, 2), (1, 2, 1.0, 1.0)),
    ((5, 5, 1), (2, 3, 0.75, 0.75)),
    ((1, 1, 1), (0, 1, 0.75, 0.75)),
    ((7, 2, 3), (1, 2, 0.25, 1.25)),
    ((9, 4, 0), (9, 4, 0.25, 0.5)),
]


@pytest.mark.parametrize("case", HAND)
def test_shima_update_hand_worked(oracle_lib, case):
    O = oracle_lib
    (xj, xk, g), want = case
    got = O.update(g, xj, xk, 0.25, 0.5)
    assert got == want
    # total droplet volume is conserved exactly with dyadic volumes
    assert got[0] * got[2] + got[1] * got[3] == xj * 0.25 + xk * 0.5
    # droplet number falls by gamma * xi_k
    assert got[0] + got[1] == xj + xk - g * xk


def test_gamma_rules(oracle_lib):
    O = oracle_lib
    assert O.gamma(0.0, 0.0, 5, 5) == 0
    assert O.gamma(0.0, 0.999, 5, 5) == 0
    assert O.gamma(0.3, 0.3, 5, 5) == 0  # p == u -> ceil(0) = 0
    assert O.gamma(0.3, 0.2999, 5, 5) == 1
    assert O.gamma(2.3, 0.0, 9, 1) == 3  # u = 0 -> ceil(p)
    assert O.gamma(2.0, 0.0, 9, 1) == 2
    assert O.gamma(5.5, 0.1, 7, 2) == 3  # capped at floor(7/2)
    assert O.gamma(1e300, 0.5, 2**62, 3) == 2**62 // 3  # no overflow


def test_gamma_frequencies_match_fractional_part(oracle_lib):
    """With u from the pair stream, gamma = ceil(p - u) is 3 w.p. frac(p)=0.3 and 2 otherwise."""
    O = oracle_lib
    u = np.array([O.pair_uniform(1, l, c, 4) for c in range(10) for l in range(5000)])
    g = np.array([O.gamma(2.3, t, 100, 1) for t in u[:20000]])
    assert set(np.unique(g)) <= {2, 3}
    frac3 = np.mean(g == 3)
    sd = math.sqrt(0.3 * 0.7 / len(g))
    assert abs(frac3 - 0.3) < 5 * sd
    # E[gamma] = p for an uncapped pair
    assert abs(g.mean() - 2.3) < 5 * sd


@pytest.mark.parametrize("n_c,factor", [(2, 1.0), (3, 3.0), (4, 3.0), (5, 5.0), (256, 255.0), (257, 257.0)])
def test_scale_factor(oracle_lib, n_c, factor):
    """[n_c (n_c - 1) / 2] / floor(n_c / 2) times dt / dV."""
    O = oracle_lib
    P = O.params(dt=2.0, dv=8.0)
    assert O.scale(P, n_c) == 0.25 * factor


def test_probability_golovin_value(oracle_lib):
    O = oracle_lib
    P = O.params("golovin", b=1500.0, dt=1.0, dv=1e6)
    vj, vk, xij = 2.0**-40, 2.0**-41, 2**30
    sc = O.scale(P, 2)
    want = 1500.0 * (vj + vk) * xij * 1e-6
    assert O.probability(P, sc, xij, vj, vk) == pytest.approx(want, rel=1e-15)


def test_probability_kfp32_hand_case(oracle_lib):
    """KFP32 mode: K and p in binary32 in the order (K xi_j) scale.  Dyadic
    inputs make every binary32 operation exact: b = 2^10, v_j = 2^-40,
    v_k = 2^-41, xi_j = 3 2^10, dt = 1, dV = 2^-10 and n_c = 2 (scale 2^10)
    give K = 3 2^-31 and p = 9 2^-11 exactly, in both precisions."""
    O = oracle_lib
    for prec in ("fp64", "kfp32"):
        P = O.params("golovin", prec, b=1024.0, dt=1.0, dv=2.0**-10)
        sc = O.scale(P, 2)
        assert sc == 1024.0
        assert O.probability(P, sc, 3 * 1024, 2.0**-40, 2.0**-41) == 9 * 2.0**-11
        # the multiplicity passed is the one that scales p (xi_j, the larger)
        assert O.probability(P, sc, 1024, 2.0**-40, 2.0**-41) == 3 * 2.0**-11


def test_probability_kfp32_rounds_each_operation_in_binary32(oracle_lib):
    """Non-dyadic inputs: the KFP32 value is the binary32 evaluation of
    (b (v_j + v_k) xi_j) scale from the binary32 images of its inputs, each
    operation rounded once (numpy float32 arithmetic, which rounds every
    operation to nearest), and differs from the binary64 value by rounding
    only."""
    O = oracle_lib
    f = np.float32
    rng = np.random.default_rng(11)
    for _ in range(200):
        vj, vk = np.exp(rng.uniform(np.log(1e-18), np.log(1e-9), 2))
        xij = int(rng.integers(1, 2**40))
        n_c = int(rng.integers(2, 5000))
        P = O.params("golovin", "kfp32", b=1500.0, dt=1.0, dv=1e6 / 3)
        sc = O.scale(P, n_c)
        K = f(1500.0) * (f(vj) + f(vk))
        want = float((K * f(xij)) * f(sc))
        assert O.probability(P, sc, xij, vj, vk) == want
        p64 = O.probability(O.params("golovin", "fp64", b=1500.0, dt=1.0, dv=1e6 / 3), sc, xij, vj, vk)
        assert want == pytest.approx(p64, rel=4 * 2.0**-24)


# Long (1974) collision efficiency by hand from its published cgs form
# E = max(4.5e4 R^2 (1 - 3e-4 / r), 1e-3) for R <= 50 um (R, r in cm), else 1:
# (R, r) in um -> E
LONG_HAND = [
    ((50.0, 10.0), 4.5e4 * 25e-6 * 0.7),        # 0.7875
    ((20.0, 10.0), 4.5e4 * 4e-6 * 0.7),         # 0.126
    ((30.0, 6.0), 4.5e4 * 9e-6 * 0.5),          # 0.2025
    ((50.0, 50.0), 4.5e4 * 25e-6 * 0.94),       # 1.0575: the published form exceeds 1 here
    ((40.0, 2.0), 1e-3),                        # 1 - 3e-4 / r < 0: the floor
    ((10.0, 3.0), 1e-3),                        # r = 3 um: 1 - c2 / r = 0 exactly
    ((50.001, 10.0), 1.0),                      # above 50 um
    ((600.0, 100.0), 1.0),
]


@pytest.mark.parametrize("case", LONG_HAND)
def test_long_efficiency_hand_values(oracle_lib, case):
    O = oracle_lib
    (R, r), want = case
    R, r = R * 1e-6, r * 1e-6
    assert O.efficiency_long(R, r) == pytest.approx(want, rel=1e-14)
    assert O.efficiency_long(r, R) == O.efficiency_long(R, r)  # symmetric in the pair
    assert O.efficiency_longf(R, r) == pytest.approx(want, rel=2e-6)


def test_long_kernel_is_geometric_times_efficiency(oracle_lib):
    """K_Long = E(r_j, r_k) K_geometric in both precisions (one extra
    rounded product), E within (1e-3, 1.125]: never above 4.5e8 R_lim^2."""
    O = oracle_lib
    Pg, Pl = O.params("geometric"), O.params("long")
    Pgf, Plf = O.params("geometric", "kfp32"), O.params("long", "kfp32")
    rng = np.random.default_rng(8)
    for _ in range(300):
        vj, vk = np.exp(rng.uniform(np.log(1e-18), np.log(1e-8), 2))
        rj, rk = O.radius(vj), O.radius(vk)
        e = O.efficiency_long(rj, rk)
        assert 1e-3 <= e <= 1.125
        assert O.kernel(Pl, vj, vk) == O.kernel(Pg, vj, vk) * e
        assert O.kernel(Pl, vk, vj) == O.kernel(Pl, vj, vk)
        kf = O.kernelf(Plf, vj, vk)
        # binary32 rounding relative to the magnitude of the terms (the speed
        # difference and 1 - c2 / r can cancel)
        R, r = max(rj, rk), min(rj, rk)
        em = 1.0 if R > 50e-6 else 4.5e8 * R * R * (1 + 3e-6 / r) + 1e-3
        mag = math.pi * (rj + rk) ** 2 * (O.vt(Pg, rj) + O.vt(Pg, rk)) * em
        assert abs(kf - O.kernel(Pl, vj, vk)) <= 1e-5 * mag + 1e-30
        assert O.kernelf(Pgf, vj, vk) * O.efficiency_longf(np.float32(O.radius(vj)), np.float32(O.radius(vk))) \
            == pytest.approx(kf, rel=1e-5, abs=1e-30)


def test_cbrt_against_libm(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(5)
    x = np.exp(rng.uniform(np.log(1e-300), np.log(1e300), 20000))
    x = np.concatenate([x, np.exp(rng.uniform(np.log(1e-31), np.log(1e-3), 20000))])
    y = O.cbrt(x)
    ref = np.cbrt(x)
    ulp = np.abs(y - ref) / np.spacing(ref)
    assert ulp.max() <= 1.0
    # perfect cubes come out exact
    for i in range(1, 2000, 7):
        for e in (-60, 0, 33):
            r = math.ldexp(float(i), e)
            assert O.cbrt(np.array([r * r * r]))[0] == r


def test_cbrtf_accuracy(oracle_lib):
    """binary32 cube root within 1 ulp of the exact value (sampled here; the
    exponent split is exact, so [1, 8) covers every binade)."""
    O = oracle_lib
    rng = np.random.default_rng(6)
    x = rng.uniform(1.0, 8.0, 30000).astype(np.float32)
    x = np.concatenate([x, np.float32(2.0) ** rng.integers(-120, 120, 500).astype(np.float32)])
    y = O.cbrtf(x).astype(np.float64)
    ref = np.cbrt(x.astype(np.float64))
    ulp = np.abs(y - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert ulp.max() <= 1.0


def test_radius_of_volume(oracle_lib):
    O = oracle_lib
    for r in (1e-6, 15e-6, 30.531e-6, 1e-3):
        v = 4.0 / 3.0 * math.pi * r**3
        assert O.radius(v) == pytest.approx(r, rel=4e-16)


def test_terminal_velocity_against_measured(oracle_lib):
    """Rogers-Yau fall speeds against Gunn & Kinzer (1949) measurements of
    drops in still air: diameter 0.02 mm -> 1.2 cm/s, 0.2 mm -> 0.72 m/s,
    1 mm -> 4.03 m/s, 2 mm -> 6.49 m/s (20 % band: the fit is piecewise)."""
    O = oracle_lib
    P = O.params("geometric")
    for d_mm, vt_meas in [(0.02, 0.012), (0.2, 0.72), (1.0, 4.03), (2.0, 6.49)]:
        r = d_mm * 1e-3 / 2
        assert O.vt(P, r) == pytest.approx(vt_meas, rel=0.2)
    # regime values at the boundaries are the published forms
    assert O.vt(P, 39.999e-6) == pytest.approx(1.19e8 * 39.999e-6**2, rel=1e-15)
    assert O.vt(P, 40e-6) == pytest.approx(8e3 * 40e-6, rel=1e-15)
    assert O.vt(P, 600e-6) == pytest.approx(201.0 * math.sqrt(600e-6), rel=1e-15)


def test_geometric_kernel_invariants(oracle_lib):
    O = oracle_lib
    P = O.params("geometric")
    rng = np.random.default_rng(7)
    for _ in range(200):
        vj, vk = np.exp(rng.uniform(np.log(1e-18), np.log(1e-8), 2))
        kj = O.kernel(P, vj, vk)
        assert kj >= 0.0
        assert kj == O.kernel(P, vk, vj)
        assert O.kernel(P, vj, vj) == 0.0
        kf = O.kernelf(P, vj, vk)
        assert kf == pytest.approx(kj, rel=1e-5, abs=1e-6 * (kj + 1e-30))
    # one hand-evaluated value: r = 100 um and 10 um
    vj = 4 / 3 * math.pi * 100e-6**3
    vk = 4 / 3 * math.pi * 10e-6**3
    want = math.pi * (110e-6) ** 2 * (8e3 * 100e-6 - 1.19e8 * 10e-6**2)
    assert O.kernel(P, vj, vk) == pytest.approx(want, rel=1e-13)
