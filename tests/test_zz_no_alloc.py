"""The allocation-free entry point (sdm_cell_step_noalloc) against the
regular context path.

Callers that cannot allocate device memory mid-run (a host model with its own
fixed pool, a Fortran/OpenACC runtime that owns every device buffer) step one
cell held in their own arrays; the library's scratch is a fixed device array.
The result must equal sdm_coalescence_step on a one-cell context with the
same config and step index, here bit for bit (the tolerance of the parity
tests), over two calls in a row.  This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm

    B.build()
    torch.cuda.set_device(0)
    return sdm, torch


def _cell(n, seed):
    rng = np.random.default_rng(seed)
    xi = np.where(rng.random(n) < 0.3, 1000, rng.integers(1, 10**9, n)).astype(np.int64)
    xi[rng.random(n) < 0.05] = 0
    r = np.exp(rng.uniform(np.log(2e-6), np.log(2e-3), n))
    return xi, 4 / 3 * np.pi * r**3


@pytest.mark.parametrize("kernel,precision,n,dv", [("golovin", "fp64", 3000, 1e-2), ("geometric", "fp64", 20000, 1e-3),
                                                   ("geometric", "kfp32", 512, 1e-3),
                                                   ("golovin", "fp64", 1 << 20, 1e2)])
def test_noalloc_equals_context_two_calls(env, kernel, precision, n, dv):
    sdm, torch = env
    xi, v = _cell(n, n)
    s0 = 41
    cfg = sdm.make_config(kernel, precision, dv=dv, n_cells=1, seed=7)
    dev = torch.device("cuda", 0)
    xi_d = torch.from_numpy(xi).to(dev)
    v_d = torch.from_numpy(v).to(dev)
    stream = sdm.current_stream_handle()
    sdm.sdm_cell_step_noalloc(cfg, s0, xi_d, v_d, stream)
    sdm.sdm_cell_step_noalloc(cfg, s0 + 1, xi_d, v_d, stream)
    torch.cuda.synchronize()
    run = sdm.Run(sdm.make_config(kernel, precision, dv=dv, n_cells=1, seed=7, step0=s0), n)
    run.set_attributes(xi, v, np.zeros(n, np.int32)).step(2)
    want_xi, want_v = run.attributes()
    run.close()
    got_xi, got_v = xi_d.cpu().numpy(), v_d.cpu().numpy()
    assert np.array_equal(got_xi, want_xi)
    assert np.array_equal(got_v, want_v)
    assert int((got_xi != xi).sum()) > 0


def test_noalloc_rejects_bad_sizes(env):
    sdm, torch = env
    dev = torch.device("cuda", 0)
    cfg = sdm.make_config("golovin", n_cells=1)
    stream = sdm.current_stream_handle()
    big = sdm.NOALLOC_MAX_SD + 2
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_step_noalloc(cfg, 0, torch.ones(big, dtype=torch.int64, device=dev),
                                  torch.ones(big, dtype=torch.float64, device=dev), stream)
    assert e.value.status == sdm.SDM_EINVAL and "SDM_NOALLOC_MAX_SD" in str(e.value)
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_step_noalloc(cfg, 0, torch.ones(7, dtype=torch.int64, device=dev),
                                  torch.ones(7, dtype=torch.float64, device=dev), stream)
    assert e.value.status == sdm.SDM_EINVAL and "even" in str(e.value)
    # a context's piece-of-grid offset has no meaning here (random streams of cell 0)
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_step_noalloc(sdm.make_config("golovin", n_cells=1, cell_base=8), 0,
                                  torch.ones(64, dtype=torch.int64, device=dev),
                                  torch.ones(64, dtype=torch.float64, device=dev), stream)
    assert e.value.status == sdm.SDM_EINVAL
    # a volume array shorter than xi is refused on the host, before any launch
    with pytest.raises(ValueError):
        sdm.sdm_cell_step_noalloc(cfg, 0, torch.ones(64, dtype=torch.int64, device=dev),
                                  torch.ones(32, dtype=torch.float64, device=dev), stream)
    # host memory handed to the C entry point directly is refused by its
    # pointer check, before any launch
    xi_h = torch.ones(64, dtype=torch.int64).pin_memory()
    v_h = torch.ones(64, dtype=torch.float64).pin_memory()
    rc = sdm.load().sdm_cell_step_noalloc(sdm.ctypes.byref(cfg), 0, sdm.ctypes.c_void_p(xi_h.data_ptr()),
                                          sdm.ctypes.c_void_p(v_h.data_ptr()), 64, sdm.ctypes.c_void_p(stream))
    assert rc == sdm.SDM_EINVAL


def test_noalloc_allocates_no_device_memory(env):
    """After a first call (the per-device set-up), further calls leave the
    device's free memory and torch's allocator untouched."""
    sdm, torch = env
    dev = torch.device("cuda", 0)
    n = 1 << 16
    xi, v = _cell(n, 3)
    cfg = sdm.make_config("geometric", dv=1e-2, n_cells=1, seed=3)
    xi_d = torch.from_numpy(xi).to(dev)
    v_d = torch.from_numpy(v).to(dev)
    stream = sdm.current_stream_handle()
    sdm.sdm_cell_step_noalloc(cfg, 0, xi_d, v_d, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    alloc0 = torch.cuda.memory_allocated(dev)
    for s in range(1, 6):
        sdm.sdm_cell_step_noalloc(cfg, s, xi_d, v_d, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert free1 == free0
