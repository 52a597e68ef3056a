"""Brute-force pins of the random permutation and of the expected collision
rate on tiny cells."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats


def test_permutation_is_sort_by_key_then_rank(oracle_lib):
    O = oracle_lib
    xi = np.array([3, 0, 5, 1, 1, 0, 9, 2], dtype=np.int64)
    perm = O.permutation(42, 7, 13, xi)
    live = [q for q in range(len(xi)) if xi[q] > 0]
    want = sorted(live, key=lambda q: (O.sort_key(42, q, 7, 13), q))
    assert list(perm) == want
    assert all(xi[q] > 0 for q in perm)


def test_order_ties_broken_by_rank(oracle_lib):
    O = oracle_lib
    assert O.order(5, 1, 5, 2) < 0 and O.order(5, 2, 5, 1) > 0
    assert O.order(4, 9, 5, 1) < 0 and O.order(2**64 - 1, 0, 2**63, 7) > 0
    assert O.order(7, 3, 7, 3) == 0


def test_permutation_uniform_n4(oracle_lib):
    """All 24 orders of 4 live SDs are equally likely."""
    O = oracle_lib
    xi = np.ones(4, dtype=np.int64)
    counts = {}
    n = 24000
    for s in range(n):
        key = tuple(O.permutation(9, 0, s, xi))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    obs = np.array([counts[p] for p in itertools.permutations(range(4))])
    assert stats.chisquare(obs).pvalue > 1e-4


def test_unpaired_uniform_n3(oracle_lib):
    O = oracle_lib
    xi = np.array([1, 0, 1, 1], dtype=np.int64)  # rank 1 dead
    left = np.zeros(4, dtype=np.int64)
    for s in range(9000):
        perm = O.permutation(5, 2, s, xi)
        assert len(perm) == 3 and 1 not in perm
        left[perm[2]] += 1
    assert left[1] == 0
    assert stats.chisquare(left[[0, 2, 3]]).pvalue > 1e-4


def _kernel_independent(kernel, vi, vj, b=1500.0):
    """K(i, j) written out from its definition in binary64 numpy, apart from
    the oracle: Golovin b (v_i + v_j), or the geometric sweep-out
    pi (r_i + r_j)^2 |v_t(r_i) - v_t(r_j)| with r = (3 v / 4 pi)^(1/3) and the
    Rogers-Yau speeds k1 r^2 (r < 40 um), k2 r (r < 600 um), k3 sqrt(r)."""
    if kernel == "golovin":
        return b * (vi + vj)

    def vt(r):
        if r < 40e-6:
            return 1.19e8 * r * r
        if r < 600e-6:
            return 8.0e3 * r
        return 201.0 * math.sqrt(r)

    ri, rj = (float(np.cbrt(3.0 * x / (4.0 * math.pi))) for x in (vi, vj))
    k = math.pi * (ri + rj) ** 2 * abs(vt(ri) - vt(rj))
    if kernel == "long":
        k *= _long_efficiency_cgs(max(ri, rj) * 100.0, min(ri, rj) * 100.0)
    return k


def _long_efficiency_cgs(R, r):
    """Long's (1974) collision efficiency in its published cgs form (radii in
    cm): max(4.5e4 R^2 (1 - 3e-4 / r), 1e-3) for R <= 50 um, else 1."""
    if R > 50e-4:
        return 1.0
    return max(4.5e4 * R * R * (1.0 - 3e-4 / r), 1e-3)


@pytest.mark.parametrize("kernel,precision", [("golovin", "fp64"), ("golovin", "kfp32"),
                                              ("geometric", "fp64"), ("geometric", "kfp32"),
                                              ("long", "fp64"), ("long", "kfp32")])
@pytest.mark.parametrize("n_c", [2, 3, 8, 9])
def test_expected_collisions_equal_mean_field_rate(oracle_lib, n_c, kernel, precision):
    """E[sum of gamma over the drawn pairs] = sum over ALL pairs i<j of
    K_ij max(xi_i, xi_j) dt/dV: the [n_c(n_c-1)/2]/floor(n_c/2) factor makes
    floor(n_c/2) random pairs stand for every pair.  Exact expectation by
    brute force over pairs, versus the mean over 4000 one-step runs.  In
    KFP32 mode K and p are binary32 (relative rounding below 1e-5 here,
    added to the statistical band); a dropped scale, p taken with the smaller
    multiplicity or a swapped operand in either precision's branch moves the
    mean by far more than the band."""
    O = oracle_lib
    rng = np.random.default_rng(n_c)
    # volumes spanning radii ~6 to ~60 um: the geometric kernel's Stokes and
    # linear regimes both occur, and Long's efficiency on both sides of 50 um
    v = np.exp(rng.uniform(np.log(1e-15), np.log(1e-12), n_c))
    xi = rng.integers(10**6, 10**7, n_c).astype(np.int64)
    pairs = [(i, j) for i in range(n_c) for j in range(i + 1, n_c)]
    kmax = max(_kernel_independent(kernel, v[i], v[j]) for i, j in pairs)
    # every p stays below 1/2: p <= K_max xi_max n_c / dV
    dv = 2.0 * kmax * float(xi.max()) * n_c
    P = O.params(kernel, precision, b=1500.0, dt=1.0, dv=dv)
    want = sum(_kernel_independent(kernel, v[i], v[j]) * max(xi[i], xi[j]) / dv for i, j in pairs)
    tot = 0
    runs = 4000
    for seed in range(runs):
        st = O.State(xi.copy(), v.copy(), np.zeros(n_c, np.int32), None, 1)
        P.seed = seed
        tot += O.step(P, st, 0).sum_gamma
    mean = tot / runs
    # gamma per pair is Bernoulli(p) with p <= 1/2 here: variance <= want
    assert abs(mean - want) < 5 * math.sqrt(want / runs) + 1e-5 * want


def _tie_fixture():
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "sort_word_ties.txt")
    return [tuple(int(t) for t in line.split()) for line in open(path) if not line.startswith("#")]


def test_keys_sharing_their_top_bits_are_ordered_by_the_full_key(oracle_lib):
    """The cells listed in golden/sort_word_ties.txt hold two keys that agree
    in their top 24 bits and order against their ranks; the permutation
    orders them by the full 64-bit key, so the later rank comes first."""
    import importlib.util
    import os

    O = oracle_lib
    spec = importlib.util.spec_from_file_location(
        "make_ties", os.path.join(os.path.dirname(__file__), "golden", "make_sort_word_ties.py"))
    M = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(M)
    rows = _tie_fixture()
    assert len(rows) >= 5
    for cell, p in rows:
        assert p in M.tie_positions(cell)
        perm = O.permutation(0, cell, 0, np.ones(256, np.int64))
        a, b = int(perm[p]), int(perm[p + 1])
        assert a > b
        ka, kb = O.sort_key(0, a, cell, 0), O.sort_key(0, b, cell, 0)
        assert ka >> 40 == kb >> 40 and ka < kb
