"""Diagnostics and failure detection on the GPU.

The conservation sums (sdm_diagnostics) against the state's own sums and the
oracle's: Shima's update conserves the total water volume sum(xi v) up to
binary64 rounding and never increases the total multiplicity sum(xi).  The
bounded-wait self-test gives up on a barrier that nothing completes and
reports SDM_ETIMEOUT, with the device usable afterwards.  A device allocator
that fails is reported as SDM_ENOMEM, without a crash or a leak of the
context."""
import ctypes
import math

import numpy as np
import pytest

from paper_2103_17238_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm

    B.build()
    O.build()
    torch.cuda.set_device(0)
    return O, sdm, torch


def _host_sums(xi, v, cell):
    inside = (cell >= 0) & (xi > 0)
    return int(inside.sum()), sum(int(x) for x in xi[inside]), math.fsum((xi[inside].astype(float) * v[inside]))


@pytest.mark.parametrize("kernel", ["geometric", "golovin"])
def test_diagnostics_conserve_and_match_the_oracle(env, kernel):
    O, sdm, torch = env
    g = I.grid_geometric(side=8, sd_per_cell=256, seed=3)
    dv = g.dv if kernel == "geometric" else 1e-2
    run = sdm.Run(sdm.make_config(kernel, dv=dv, n_cells=g.n_cells, seed=4), g.n_sd)
    run.set_attributes(g.xi, g.v, g.cell)
    d0 = run.diagnostics()
    live, sxi, sxv = _host_sums(g.xi, g.v, g.cell)
    assert d0["live_sd"] == live and d0["sum_xi"] == sxi
    assert math.isclose(d0["sum_xi_v"], sxv, rel_tol=1e-13)
    assert run.diagnostics() == d0  # the same bits again
    run.step(200)
    d1 = run.diagnostics()
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, g.n_cells)
    O.run(O.params(kernel, dv=dv, seed=4), st, 0, 200)
    live1, sxi1, sxv1 = _host_sums(st.xi, st.v, st.cell)
    assert d1["live_sd"] == live1 and d1["sum_xi"] == sxi1
    assert sxi1 < sxi  # collisions took place, and the multiplicity only fell
    assert math.isclose(d1["sum_xi_v"], sxv1, rel_tol=1e-13)
    assert math.isclose(d1["sum_xi_v"], d0["sum_xi_v"], rel_tol=1e-12)  # water conserved
    run.close()


def test_diagnostics_count_only_the_domain_and_exact_big_sums(env):
    O, sdm, torch = env
    n = 4096
    rng = np.random.default_rng(9)
    cell = rng.integers(-1, 4, n).astype(np.int32)          # some SDs outside the domain
    xi = rng.integers(2**60, 2**62, n).astype(np.int64)     # the sum needs more than 64 bits
    xi[rng.random(n) < 0.1] = 0
    v = 4 / 3 * np.pi * np.exp(rng.uniform(np.log(3e-6), np.log(3e-4), n)) ** 3
    run = sdm.Run(sdm.make_config("golovin", dv=1e6, n_cells=4), n).set_attributes(xi, v, cell)
    d = run.diagnostics()
    live, sxi, sxv = _host_sums(xi, v, cell)
    assert d["live_sd"] == live and d["sum_xi"] == sxi and sxi > 2**64
    assert math.isclose(d["sum_xi_v"], sxv, rel_tol=1e-13)
    run.close()


def test_bounded_wait_gives_up_and_the_device_stays_usable(env):
    O, sdm, torch = env
    stream = torch.cuda.current_stream().cuda_stream
    for polls in (1, 64, 4096):
        assert sdm.sdm_selftest_bounded_wait(polls, stream) == sdm.SDM_ETIMEOUT
        assert b"as designed" in sdm.load().sdm_last_error(None)
    g = I.box_golovin(512, seed=0)
    run = sdm.Run(sdm.make_config("golovin", dv=g.dv, seed=0), g.n_sd).set_attributes(g.xi, g.v, g.cell)
    run.step(5)
    st = O.State(g.xi.copy(), g.v.copy(), g.cell.copy(), None, 1)
    O.run(O.params("golovin", dv=g.dv, seed=0), st, 0, 5)
    xi, v = run.attributes()
    assert np.array_equal(xi, st.xi) and np.array_equal(v, st.v)
    run.close()


def test_failing_device_allocator_is_reported(env):
    O, sdm, torch = env
    keep = []

    def make_cfg(fail_after):
        calls = {"n": 0}
        live = {}

        def alloc(nbytes, stream, user):
            calls["n"] += 1
            if calls["n"] > fail_after:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
            live[p] = nbytes
            return p

        def free(ptr, nbytes, stream, user):
            if ptr:
                live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)

        cfg = sdm.make_config("golovin", dv=1e6, seed=0)
        fa, ff = sdm.ALLOC_FN(alloc), sdm.FREE_FN(free)
        keep.extend([fa, ff])
        cfg.alloc, cfg.free = fa, ff
        return cfg, calls, live

    stream = torch.cuda.current_stream().cuda_stream
    cfg, calls, live = make_cfg(0)  # nothing can be allocated
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_create(cfg, 4096, stream)
    assert e.value.status == sdm.SDM_ENOMEM and not live

    cfg, calls, live = make_cfg(10**9)  # count what creating a context takes
    h = sdm.sdm_create(cfg, 4096, stream)
    n_create = calls["n"]
    sdm.sdm_destroy(h)
    torch.cuda.synchronize()
    assert not live

    g = I.box_golovin(4096, seed=1)
    cfg, calls, live = make_cfg(n_create)  # the context, then nothing more
    h = sdm.sdm_create(cfg, 4096, stream)
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_set_attributes(h, g.xi, g.v, g.cell)
    assert e.value.status == sdm.SDM_ENOMEM
    sdm.sdm_destroy(h)
    torch.cuda.synchronize()
    assert not live
