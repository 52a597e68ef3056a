"""Invariants of the oracle over whole runs: total droplet volume conserved,
total number non-increasing, multiplicities non-negative, step-index
addressing (resume), and instance i of seed S equal to a lone run with seed
S + i."""
import math

import numpy as np
import pytest

from paper_2103_17238_gb300 import inputs as I


def _state(O, inst):
    return O.State(inst.xi.copy(), inst.v.copy(), inst.cell.copy(), None, inst.n_cells)


@pytest.mark.parametrize("kernel,precision", [("golovin", "fp64"), ("geometric", "fp64"),
                                              ("geometric", "kfp32"), ("golovin", "kfp32"),
                                              ("long", "fp64"), ("long", "kfp32")])
def test_conservation_and_monotone_number(oracle_lib, kernel, precision):
    O = oracle_lib
    inst = I.grid_geometric(side=4, sd_per_cell=64) if kernel != "golovin" else I.box_golovin(512)
    P = O.params(kernel, precision, dv=inst.dv)
    st = _state(O, inst)
    vol0 = math.fsum(st.xi * st.v)
    n_prev = int(st.xi.sum())
    colls = 0
    for s in range(300):
        colls += O.step(P, st, s).n_collisions
        assert st.xi.min() >= 0
        assert np.all(st.v > 0)
        n = int(st.xi.sum())
        assert n <= n_prev
        n_prev = n
    assert colls > 0
    assert abs(math.fsum(st.xi * st.v) - vol0) <= 1e-12 * vol0


def test_resume_by_step_index(oracle_lib):
    O = oracle_lib
    inst = I.grid_geometric(side=3, sd_per_cell=32)
    P = O.params("geometric", dv=inst.dv, seed=77)
    a = _state(O, inst)
    O.run(P, a, 0, 40)
    b = _state(O, inst)
    O.run(P, b, 0, 17)
    O.run(P, b, 17, 23)
    assert np.array_equal(a.xi, b.xi) and np.array_equal(a.v, b.v)


def test_instance_is_seed_offset(oracle_lib):
    O = oracle_lib
    insts = [I.box_golovin(n, seed=i) for i, n in enumerate([40, 64, 9])]
    xi = np.concatenate([t.xi for t in insts])
    v = np.concatenate([t.v for t in insts])
    cell = np.zeros(len(xi), np.int32)
    inst = np.concatenate([np.full(t.n_sd, i, np.int32) for i, t in enumerate(insts)])
    both = O.State(xi.copy(), v.copy(), cell, inst, 1, 3)
    P = O.params("golovin", dv=1e6 * 1e-4, seed=10)
    O.run(P, both, 0, 25)
    off = 0
    for i, t in enumerate(insts):
        alone = O.State(t.xi.copy(), t.v.copy(), t.cell, None, 1)
        Pi = O.params("golovin", dv=1e6 * 1e-4, seed=10 + i)
        O.run(Pi, alone, 0, 25)
        assert np.array_equal(alone.xi, both.xi[off:off + t.n_sd])
        assert np.array_equal(alone.v, both.v[off:off + t.n_sd])
        off += t.n_sd


def test_dead_sds_drop_out(oracle_lib):
    """With xi = 1 everywhere every collision kills an SD (split of 1 -> 0 + 1)."""
    O = oracle_lib
    n = 64
    st = O.State(np.ones(n, np.int64), np.full(n, 1e-12), np.zeros(n, np.int32), None, 1)
    P = O.params("golovin", b=1500.0, dv=1e-9)  # p >> 1: every pair collides
    O.step(P, st, 0)
    assert int((st.xi == 0).sum()) == n // 2
    O.step(P, st, 1)
    assert int((st.xi == 0).sum()) == n // 2 + n // 4
    assert math.isclose(math.fsum(st.xi * st.v), n * 1e-12, rel_tol=1e-14)
