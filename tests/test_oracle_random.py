"""Pins of the oracle's random numbers: Philox4x32-10 against its published
known-answer vectors and an independent pure-Python rendering of the SC'11
definition; the counter layout; the distribution of u."""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def _philox_py(ctr, key, rounds=10):
    """Philox4x32 from the SC'11 paper: per round two 32x32->64 products
    (multipliers 0xD2511F53, 0xCD9E8D57), output words permuted and xored with
    the round key; keys bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85."""
    M = 0xFFFFFFFF
    x = list(ctr)
    k = list(key)
    for r in range(rounds):
        if r:
            k = [(k[0] + 0x9E3779B9) & M, (k[1] + 0xBB67AE85) & M]
        p0 = 0xD2511F53 * x[0]
        p1 = 0xCD9E8D57 * x[2]
        x = [((p1 >> 32) ^ x[1] ^ k[0]) & M, p1 & M, ((p0 >> 32) ^ x[3] ^ k[1]) & M, p0 & M]
    return x


def test_philox_known_answers(oracle_lib):
    O = oracle_lib
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(O.philox4x32_10(ctr, key)) == want
        assert _philox_py(ctr, key) == want


def test_philox_matches_independent_rendering(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(11)
    for _ in range(300):
        ctr = [int(t) for t in rng.integers(0, 2**32, 4)]
        key = [int(t) for t in rng.integers(0, 2**32, 2)]
        assert list(O.philox4x32_10(ctr, key)) == _philox_py(ctr, key)


@pytest.mark.parametrize("s", [0, 7, 2**32 + 5, 2**62 + 3])
def test_counter_layout(oracle_lib, s):
    """Sort keys use tag 0, pair uniforms tag 1; index >> 1 in word 0, the cell
    in word 1, the step split over words 2 and 3; even index -> words (0,1)."""
    O = oracle_lib
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    lo, hi = s & 0xFFFFFFFF, (s >> 32) & 0x7FFFFFFF
    for idx, cell in [(0, 0), (1, 0), (6, 3), (7, 3), (1001, 65535)]:
        w = _philox_py([idx >> 1, cell, lo, hi], key)
        a, b = (w[2], w[3]) if idx & 1 else (w[0], w[1])
        assert O.sort_key(seed, idx, cell, s) == (a << 32) | b
        w = _philox_py([idx >> 1, cell, lo, hi | (1 << 31)], key)
        a, b = (w[2], w[3]) if idx & 1 else (w[0], w[1])
        m = (a << 21) | (b >> 11)
        assert O.pair_uniform(seed, idx, cell, s) == m * 2.0**-53


def test_pair_uniform_distribution(oracle_lib):
    O = oracle_lib
    u = np.array([O.pair_uniform(3, l, c, 11) for c in range(20) for l in range(2000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    # 53-bit dyadic rationals
    assert np.all(u * 2.0**53 == np.floor(u * 2.0**53))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
