"""The continuous-batching server: runs of mixed kind, size, length and dt
are admitted under a device-memory budget as memory frees up, stepped
together, and each result equals the same run stepped alone, bit for bit."""
import numpy as np
import pytest

from paper_2103_17238_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm, serve

    B.build()
    torch.cuda.set_device(0)
    return sdm, serve, torch


def _stream(n=14):
    reqs = I.serving_stream(n_requests=n, rate=400.0, rng_seed=11, lo_log2=8.0, hi_log2=13.0)
    for i, r in enumerate(reqs):
        r.inst.steps = 20 + 7 * (i % 5)
    return reqs


@pytest.mark.parametrize("fuse", [None, 0, 8])
def test_served_equals_alone(env, fuse):
    """With the process-wide tuning, with one launch per step, and with each
    tick's steps fused for the small cells; the tuning is restored after
    every batch is built."""
    sdm, serve, torch = env
    reqs = _stream()
    fps = [serve.footprint(r.inst) for r in reqs]
    budget = 3 * max(fps)  # forces queueing: only a few runs fit at once
    srv = serve.Server(budget, chunk=8, keep_state=True, time_scale=1.0, fuse_steps=fuse)
    before = sdm.sdm_get_tuning()
    out = srv.serve(reqs)
    assert sdm.sdm_get_tuning() == before
    assert out["requests"] == len(reqs)
    assert out["step_latency_ms"]["p99"] is not None
    # admission respected the budget, and runs overlapped on the device
    assert out["max_used_bytes"] <= budget
    assert out["max_active"] > 1
    for s in out["served"]:
        run = serve.make_run(s.req.inst)
        run.step(s.req.inst.steps)
        xi, v = run.attributes()
        spec = run.spectrum(I.R_EDGES)
        run.close()
        assert np.array_equal(xi, s.xi) and np.array_equal(v, s.v)
        assert np.array_equal(spec, s.spectrum) or np.allclose(spec, s.spectrum, rtol=1e-12, atol=0)


def test_over_budget_request_rejected(env):
    sdm, serve, torch = env
    reqs = _stream(2)
    with pytest.raises(sdm.SdmError) as e:
        serve.Server(16).serve(reqs)
    assert e.value.status == sdm.SDM_EBUDGET
