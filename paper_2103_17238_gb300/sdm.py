"""Python binding of the SDM coalescence library (``include/sdm.h``).

Argument marshalling only: every step of the coalescence path runs in the
CUDA kernels of ``_lib/libsdm.so``.  PyTorch supplies device memory (its
caching allocator, through the library's allocator hooks) and CUDA streams.
The functions keep the C names; ``Run`` and ``Batch`` are thin owners.

Importing this module does not need a GPU; loading the library does need
the built ``libsdm.so`` and fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsdm.so")

SDM_OK, SDM_EINVAL, SDM_ENOMEM, SDM_ECUDA, SDM_ESTATE, SDM_ETIMEOUT, SDM_EBUDGET = range(7)
STATUS_NAMES = ["SDM_OK", "SDM_EINVAL", "SDM_ENOMEM", "SDM_ECUDA", "SDM_ESTATE", "SDM_ETIMEOUT", "SDM_EBUDGET"]
KERNELS = {"golovin": 0, "geometric": 1, "long": 2}
PRECISIONS = {"fp64": 0, "kfp32": 1}

# every symbol include/sdm.h declares
EXPORTS = [
    "sdm_config_default", "sdm_create", "sdm_set_attributes", "sdm_coalescence_step", "sdm_spectrum",
    "sdm_get_attributes", "sdm_get_info", "sdm_footprint_bytes", "sdm_destroy", "sdm_last_error",
    "sdm_batch_create", "sdm_batch_step", "sdm_batch_destroy", "sdm_batch_last_error",
    "sdm_cell_step_noalloc", "sdm_set_tuning", "sdm_get_tuning",
    "sdm_set_positions", "sdm_sedimentation_step", "sdm_get_positions", "sdm_condensation_step",
    "sdm_set_heights", "sdm_get_heights",
    "sdm_diagnostics", "sdm_selftest_bounded_wait",
]
NOALLOC_MAX_SD = 1 << 20

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class SdmError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")
        self.status = status


class sdm_config(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("golovin_b", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("dv", ctypes.c_double),
        ("ry_k1", ctypes.c_double),
        ("ry_k2", ctypes.c_double),
        ("ry_k3", ctypes.c_double),
        ("ry_r1", ctypes.c_double),
        ("ry_r2", ctypes.c_double),
        ("n_cells", ctypes.c_int32),
        ("cell_base", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("step0", ctypes.c_int64),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
    ]


FUSE_STEPS_DEFAULT = 64  # SDM_FUSE_STEPS_DEFAULT of the header
MID_MAX_SD_DEFAULT = 16384  # SDM_MID_MAX_SD_DEFAULT of the header


class sdm_tuning(ctypes.Structure):
    _fields_ = [
        ("smem_max_sd", ctypes.c_int32),
        ("warp_cell_max", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("fuse_steps", ctypes.c_int32),
        ("mid_max_sd", ctypes.c_int32),
    ]


class sdm_info(ctypes.Structure):
    _fields_ = [
        ("n_sd", ctypes.c_int64),
        ("capacity_sd", ctypes.c_int64),
        ("step", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("n_cells", ctypes.c_int32),
        ("largest_cell", ctypes.c_int32),
    ]


class sdm_diag(ctypes.Structure):
    _fields_ = [
        ("live_sd", ctypes.c_int64),
        ("sum_xi_lo", ctypes.c_uint64),
        ("sum_xi_hi", ctypes.c_uint64),
        ("sum_xi_v", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libsdm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                              "(the SDM path has no CPU fallback)")
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        L.sdm_config_default.argtypes = [P(sdm_config)]
        L.sdm_config_default.restype = None
        L.sdm_create.argtypes = [P(sdm_config), i64, vp, P(vp)]
        L.sdm_set_attributes.argtypes = [vp, i64, vp, vp, vp, ctypes.c_int]
        L.sdm_coalescence_step.argtypes = [vp, i32]
        L.sdm_spectrum.argtypes = [vp, P(ctypes.c_double), i32, ctypes.c_int, vp, ctypes.c_int]
        L.sdm_get_attributes.argtypes = [vp, vp, vp, ctypes.c_int]
        L.sdm_get_info.argtypes = [vp, P(sdm_info)]
        L.sdm_footprint_bytes.argtypes = [i64, i32, i32]
        L.sdm_footprint_bytes.restype = i64
        L.sdm_destroy.argtypes = [vp]
        L.sdm_last_error.argtypes = [vp]
        L.sdm_last_error.restype = ctypes.c_char_p
        L.sdm_batch_create.argtypes = [P(vp), i32, vp, i32, i32, P(vp)]
        L.sdm_batch_step.argtypes = [vp, i32]
        L.sdm_batch_destroy.argtypes = [vp]
        L.sdm_batch_last_error.argtypes = [vp]
        L.sdm_batch_last_error.restype = ctypes.c_char_p
        L.sdm_cell_step_noalloc.argtypes = [P(sdm_config), i64, vp, vp, i64, vp]
        L.sdm_set_tuning.argtypes = [P(sdm_tuning)]
        L.sdm_set_positions.argtypes = [vp, vp, i32, ctypes.c_double, ctypes.c_int]
        L.sdm_sedimentation_step.argtypes = [vp, P(ctypes.c_double)]
        L.sdm_condensation_step.argtypes = [vp, vp, vp, ctypes.c_double, vp, ctypes.c_int]
        L.sdm_get_positions.argtypes = [vp, vp, vp, ctypes.c_int]
        L.sdm_set_heights.argtypes = [vp, vp, i32, ctypes.c_double, ctypes.c_int]
        L.sdm_get_heights.argtypes = [vp, vp, vp, ctypes.c_int]
        L.sdm_get_tuning.argtypes = [P(sdm_tuning)]
        L.sdm_diagnostics.argtypes = [vp, P(sdm_diag)]
        L.sdm_selftest_bounded_wait.argtypes = [vp, i64]
        for name in ("sdm_create", "sdm_set_attributes", "sdm_coalescence_step", "sdm_spectrum",
                     "sdm_get_attributes", "sdm_get_info", "sdm_destroy", "sdm_batch_create",
                     "sdm_batch_step", "sdm_batch_destroy", "sdm_cell_step_noalloc", "sdm_set_tuning",
                     "sdm_get_tuning", "sdm_set_positions", "sdm_sedimentation_step", "sdm_get_positions",
                     "sdm_diagnostics", "sdm_selftest_bounded_wait"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(st: int, where: str, ctx=None, batch=None):
    if st != SDM_OK:
        L = load()
        msg = (L.sdm_batch_last_error(batch) if batch is not None else L.sdm_last_error(ctx)) or b""
        raise SdmError(st, where, msg.decode(errors="replace"))


# --------------------------------------------------------- torch plumbing
def _torch():
    import torch

    return torch


class _TorchAllocator:
    """Routes the library's device allocations to torch's caching allocator."""

    def __init__(self, device: int):
        torch = _torch()
        self.device = device
        self.sizes = {}

        def alloc(nbytes, stream, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            except Exception:
                return None
            return p

        def free(ptr, nbytes, stream, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


def current_stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr_and_flag(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=dtype)
        return a.ctypes.data, 0, a
    torch = _torch()
    if isinstance(a, torch.Tensor):
        tdt = {np.int64: torch.int64, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        a = a.contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0, a
    a = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    return a.ctypes.data, 0, a


# ------------------------------------------------------------- C names
def sdm_config_default() -> sdm_config:
    cfg = sdm_config()
    load().sdm_config_default(ctypes.byref(cfg))
    return cfg


def sdm_create(cfg: sdm_config, capacity_sd: int, stream: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().sdm_create(ctypes.byref(cfg), int(capacity_sd), ctypes.c_void_p(stream), ctypes.byref(h)),
           "sdm_create")
    return h


def sdm_set_attributes(ctx, xi, volume, cell_id):
    px, dx, kx = _ptr_and_flag(xi, np.int64)
    pv, dvv, kv = _ptr_and_flag(volume, np.float64)
    pc, dc, kc = _ptr_and_flag(cell_id, np.int32)
    if not (dx == dvv == dc):
        raise ValueError("xi, volume and cell_id must all be on the host or all on the device")
    n = int(kx.shape[0])
    if kv.shape[0] != n or kc.shape[0] != n:
        raise ValueError("xi, volume and cell_id must have the same length")
    _check(load().sdm_set_attributes(ctx, n, px, pv, pc, dx), "sdm_set_attributes", ctx)


def sdm_coalescence_step(ctx, n_steps: int = 1):
    _check(load().sdm_coalescence_step(ctx, int(n_steps)), "sdm_coalescence_step", ctx)


def sdm_spectrum(ctx, r_edges, per_cell: bool = False, out=None, n_cells: int | None = None):
    """dv/dlnr; returns a numpy array (out=None) or fills a device tensor."""
    e = np.ascontiguousarray(r_edges, dtype=np.float64)
    nb = len(e) - 1
    if out is None:
        if per_cell and n_cells is None:
            n_cells = sdm_get_info(ctx).n_cells
        host = np.zeros(n_cells * nb if per_cell else nb, dtype=np.float64)
        _check(load().sdm_spectrum(ctx, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(e),
                                   int(bool(per_cell)), host.ctypes.data, 0), "sdm_spectrum", ctx)
        return host.reshape(n_cells, nb) if per_cell else host
    po, on_dev, keep = _ptr_and_flag(out, np.float64)
    _check(load().sdm_spectrum(ctx, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(e),
                               int(bool(per_cell)), po, on_dev), "sdm_spectrum", ctx)
    return out


def sdm_get_attributes(ctx, n_sd: int | None = None, xi=None, volume=None):
    """Multiplicities and volumes in SD-id order (numpy, or into given tensors)."""
    if xi is None and volume is None:
        n = int(n_sd if n_sd is not None else sdm_get_info(ctx).n_sd)
        xi = np.zeros(n, dtype=np.int64)
        volume = np.zeros(n, dtype=np.float64)
        _check(load().sdm_get_attributes(ctx, xi.ctypes.data, volume.ctypes.data, 0), "sdm_get_attributes", ctx)
        return xi, volume
    px, dx, _ = _ptr_and_flag(xi, np.int64) if xi is not None else (None, None, None)
    pv, dv_, _ = _ptr_and_flag(volume, np.float64) if volume is not None else (None, None, None)
    on = dx if dx is not None else dv_
    _check(load().sdm_get_attributes(ctx, px, pv, on), "sdm_get_attributes", ctx)
    return xi, volume


def sdm_get_info(ctx) -> sdm_info:
    info = sdm_info()
    _check(load().sdm_get_info(ctx, ctypes.byref(info)), "sdm_get_info", ctx)
    return info


def sdm_diagnostics(ctx) -> dict:
    """Conservation sums of the current state: live SDs, sum of xi (exact
    int), sum of xi v (m^3)."""
    d = sdm_diag()
    _check(load().sdm_diagnostics(ctx, ctypes.byref(d)), "sdm_diagnostics", ctx=ctx)
    return {"live_sd": int(d.live_sd), "sum_xi": (int(d.sum_xi_hi) << 64) | int(d.sum_xi_lo),
            "sum_xi_v": float(d.sum_xi_v)}


def sdm_selftest_bounded_wait(max_polls: int, stream: int = 0) -> int:
    """Runs the device's bounded-wait path on a barrier nothing completes;
    returns the status (SDM_ETIMEOUT is the expected, healthy result)."""
    st = load().sdm_selftest_bounded_wait(ctypes.c_void_p(stream or None), int(max_polls))
    return int(st)


def sdm_footprint_bytes(capacity_sd: int, n_cells: int, largest_cell: int) -> int:
    return int(load().sdm_footprint_bytes(int(capacity_sd), int(n_cells), int(largest_cell)))


def sdm_destroy(ctx):
    if ctx:
        _check(load().sdm_destroy(ctx), "sdm_destroy")


def sdm_batch_create(ctxs, stream: int, use_graph: bool = False, graph_steps: int = 16):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    h = ctypes.c_void_p()
    _check(load().sdm_batch_create(arr, len(ctxs), ctypes.c_void_p(stream), int(bool(use_graph)),
                                   int(graph_steps), ctypes.byref(h)), "sdm_batch_create")
    return h


def sdm_batch_step(batch, n_steps: int = 1):
    _check(load().sdm_batch_step(batch, int(n_steps)), "sdm_batch_step", batch=batch)


def sdm_batch_destroy(batch):
    if batch:
        _check(load().sdm_batch_destroy(batch), "sdm_batch_destroy")


def sdm_cell_step_noalloc(cfg: sdm_config, step: int, xi, volume, stream: int):
    """One step of one cell held in caller device tensors (int64 xi, float64
    volume), in place, without any device allocation by the library."""
    px, dx, kx = _ptr_and_flag(xi, np.int64)
    pv, dv_, kv = _ptr_and_flag(volume, np.float64)
    if not (dx and dv_):
        raise ValueError("xi and volume must be device tensors")
    if kx.data_ptr() != xi.data_ptr() or kv.data_ptr() != volume.data_ptr():
        raise ValueError("xi and volume must be contiguous (the step works in place)")
    # the C call takes one length for both arrays and runs on the current
    # device: a shorter volume array or another device's tensor would be
    # accessed out of bounds there, so both are refused here
    if volume.numel() != xi.numel() or xi.dim() != 1 or volume.dim() != 1:
        raise ValueError("xi and volume must be 1-D with the same number of elements")
    torch = _torch()
    if xi.device != volume.device or xi.device.index != torch.cuda.current_device():
        raise ValueError("xi and volume must both be on the current CUDA device")
    _check(load().sdm_cell_step_noalloc(ctypes.byref(cfg), int(step), px, pv, int(kx.shape[0]),
                                        ctypes.c_void_p(stream)), "sdm_cell_step_noalloc")


def sdm_condensation_step(ctx, G, s, r_min: float, want_condensed: bool = True, n_cells: int | None = None,
                          out=None):
    """One condensation step; G, s: per-cell growth coefficient (m^2 s^-1)
    and supersaturation (host arrays).  Returns the per-cell condensed water
    sum(xi dV) (numpy, or `out` filled on the device) or None."""
    Ga = np.ascontiguousarray(G, dtype=np.float64)
    sa = np.ascontiguousarray(s, dtype=np.float64)
    nc = int(n_cells if n_cells is not None else sdm_get_info(ctx).n_cells)
    if Ga.shape != (nc,) or sa.shape != (nc,):
        raise ValueError("G and s need one value per cell")
    if out is not None:
        po, on_dev, _ = _ptr_and_flag(out, np.float64)
        res, flag = out, on_dev
    elif want_condensed:
        res = np.zeros(nc, dtype=np.float64)
        po, flag = res.ctypes.data, 0
    else:
        res, po, flag = None, None, 0
    _check(load().sdm_condensation_step(ctx, Ga.ctypes.data, sa.ctypes.data, float(r_min), po, flag),
           "sdm_condensation_step", ctx)
    return res


def sdm_set_positions(ctx, z, nx: int, dz: float):
    pz, dev, kz = _ptr_and_flag(z, np.float64)
    _check(load().sdm_set_positions(ctx, pz, int(nx), float(dz), dev), "sdm_set_positions", ctx)


def sdm_sedimentation_step(ctx) -> float:
    """One sedimentation step; returns the precipitated volume sum(xi v), m^3."""
    out = ctypes.c_double(0.0)
    _check(load().sdm_sedimentation_step(ctx, ctypes.byref(out)), "sdm_sedimentation_step", ctx)
    return out.value


def sdm_get_positions(ctx, n_sd: int | None = None, z=None, cell=None, want_z: bool = True):
    """Heights above the domain bottom and cells (-1: outside) in SD-id order
    (numpy, or into given tensors)."""
    if z is None and cell is None:
        n = int(n_sd if n_sd is not None else sdm_get_info(ctx).n_sd)
        zz = np.zeros(n, dtype=np.float64) if want_z else None
        cc = np.zeros(n, dtype=np.int32)
        _check(load().sdm_get_positions(ctx, zz.ctypes.data if want_z else None, cc.ctypes.data, 0),
               "sdm_get_positions", ctx)
        return zz, cc
    pz, dz_, _ = _ptr_and_flag(z, np.float64) if z is not None else (None, None, None)
    pc, dc, _ = _ptr_and_flag(cell, np.int32) if cell is not None else (None, None, None)
    on = dz_ if dz_ is not None else dc
    _check(load().sdm_get_positions(ctx, pz, pc, on), "sdm_get_positions", ctx)
    return z, cell


def sdm_set_heights(ctx, zeta, nx: int, dz: float):
    pz, dev, kz = _ptr_and_flag(zeta, np.float64)
    _check(load().sdm_set_heights(ctx, pz, int(nx), float(dz), dev), "sdm_set_heights", ctx)


def sdm_get_heights(ctx, n_sd: int | None = None):
    """(zeta, cell) in SD-id order: heights above the cells' bottoms and the
    cells in the whole grid (see include/sdm.h), numpy."""
    n = int(n_sd if n_sd is not None else sdm_get_info(ctx).n_sd)
    zz = np.zeros(n, dtype=np.float64)
    cc = np.zeros(n, dtype=np.int32)
    _check(load().sdm_get_heights(ctx, zz.ctypes.data, cc.ctypes.data, 0), "sdm_get_heights", ctx)
    return zz, cc


def sdm_set_tuning(tuning=None):
    """tuning: dict with smem_max_sd, warp_cell_max, warps_per_block and
    optionally fuse_steps (absent: the default, FUSE_STEPS_DEFAULT steps per
    fused launch; 0: one launch per step); None: defaults."""
    if tuning is None:
        _check(load().sdm_set_tuning(None), "sdm_set_tuning")
        return
    t = sdm_tuning(int(tuning["smem_max_sd"]), int(tuning["warp_cell_max"]), int(tuning["warps_per_block"]),
                   int(tuning.get("fuse_steps", FUSE_STEPS_DEFAULT)), int(tuning.get("mid_max_sd", MID_MAX_SD_DEFAULT)))
    _check(load().sdm_set_tuning(ctypes.byref(t)), "sdm_set_tuning")


def sdm_get_tuning() -> dict:
    t = sdm_tuning()
    _check(load().sdm_get_tuning(ctypes.byref(t)), "sdm_get_tuning")
    return {"smem_max_sd": t.smem_max_sd, "warp_cell_max": t.warp_cell_max, "warps_per_block": t.warps_per_block,
            "fuse_steps": t.fuse_steps, "mid_max_sd": t.mid_max_sd}


# ------------------------------------------------------------ owners
def make_config(kernel="golovin", precision="fp64", *, b=1500.0, dt=1.0, dv=1.0e6, n_cells=1, seed=0,
                step0=0, cell_base=0, **ry) -> sdm_config:
    cfg = sdm_config_default()
    cfg.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.golovin_b = b
    cfg.dt = dt
    cfg.dv = dv
    cfg.n_cells = n_cells
    cfg.seed = seed
    cfg.step0 = step0
    cfg.cell_base = cell_base
    for k, v in ry.items():
        setattr(cfg, "ry_" + k, v)
    return cfg


class Run:
    """One coalescence run on the current CUDA device and stream."""

    def __init__(self, cfg: sdm_config, capacity_sd: int, stream=None, torch_memory: bool = True):
        torch = _torch()
        self._alloc = None
        if torch_memory:
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            cfg.alloc = self._alloc.alloc
            cfg.free = self._alloc.free
        self.cfg = cfg
        self.stream = current_stream_handle(stream)
        self.h = sdm_create(cfg, capacity_sd, self.stream)

    def set_attributes(self, xi, volume, cell_id):
        sdm_set_attributes(self.h, xi, volume, cell_id)
        return self

    def step(self, n_steps: int = 1):
        sdm_coalescence_step(self.h, n_steps)
        return self

    def spectrum(self, r_edges, per_cell=False, out=None):
        return sdm_spectrum(self.h, r_edges, per_cell, out, n_cells=self.cfg.n_cells)

    def attributes(self):
        return sdm_get_attributes(self.h)

    def condense(self, G, s, r_min: float, want_condensed: bool = True):
        """One condensation step; returns the per-cell condensed water, m^3."""
        return sdm_condensation_step(self.h, G, s, r_min, want_condensed, n_cells=self.cfg.n_cells)

    def set_positions(self, z, nx: int, dz: float):
        sdm_set_positions(self.h, z, nx, dz)
        return self

    def sediment(self) -> float:
        """One sedimentation step; returns the precipitated volume, m^3."""
        return sdm_sedimentation_step(self.h)

    def positions(self, want_z: bool = True):
        return sdm_get_positions(self.h, want_z=want_z)

    def info(self) -> sdm_info:
        return sdm_get_info(self.h)

    def diagnostics(self) -> dict:
        return sdm_diagnostics(self.h)

    def close(self):
        if self.h:
            sdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several runs advanced by fused launches (optionally a CUDA graph)."""

    def __init__(self, runs, stream=None, use_graph=False, graph_steps=16):
        self.runs = list(runs)
        self.stream = current_stream_handle(stream)
        self.h = sdm_batch_create([r.h for r in self.runs], self.stream, use_graph, graph_steps)

    def step(self, n_steps: int = 1):
        sdm_batch_step(self.h, n_steps)
        return self

    def close(self):
        if self.h:
            sdm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
