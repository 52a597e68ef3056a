"""ctypes front end of the plain C SDM oracle (``sdm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never links, loads or calls it, and the two share no
source: this file only compiles the C oracle with gcc and marshals numpy
arrays in and out of it.

State convention: SDs are identified by their index in the arrays (the SD id).
``cell[i]`` is the cell of SD i within its instance, ``inst[i]`` its instance
(or ``None`` for a single instance).  Within a cell an SD's rank is its
position among that cell's SDs in increasing id, dead SDs included.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sdm_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

# IEEE binary64/binary32 with round-to-nearest and no FMA contraction is part
# of the oracle's definition (gcc on aarch64 contracts by default).
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(LIB_PATH)) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC)
    if force or stale:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("b", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("dv", ctypes.c_double),
        ("k1", ctypes.c_double),
        ("k2", ctypes.c_double),
        ("k3", ctypes.c_double),
        ("r1", ctypes.c_double),
        ("r2", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_pairs", ctypes.c_int64),
        ("n_collisions", ctypes.c_int64),
        ("sum_gamma", ctypes.c_int64),
    ]


# Rogers & Yau (1989) terminal-velocity coefficients in SI units:
# k1 = 1.19e6 cm^-1 s^-1, k2 = 8e3 s^-1, k3 = 2.01e3 cm^1/2 s^-1; regimes split
# at 40 um and 600 um.
RY_DEFAULTS = dict(k1=1.19e8, k2=8.0e3, k3=201.0, r1=40.0e-6, r2=600.0e-6)

KERNELS = {"golovin": 0, "geometric": 1, "long": 2}
PRECISIONS = {"fp64": 0, "kfp32": 1}


def params(kernel="golovin", precision="fp64", b=1500.0, dt=1.0, dv=1.0e6, seed=0, **ry) -> Params:
    c = dict(RY_DEFAULTS)
    c.update(ry)
    return Params(
        KERNELS[kernel] if isinstance(kernel, str) else int(kernel),
        PRECISIONS[precision] if isinstance(precision, str) else int(precision),
        b, dt, dv, c["k1"], c["k2"], c["k3"], c["r1"], c["r2"], seed,
    )


_P = ctypes.POINTER
_i64p = _P(ctypes.c_int64)
_i32p = _P(ctypes.c_int32)
_f64p = _P(ctypes.c_double)
_u32p = _P(ctypes.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_sort_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64]
            L.orc_sort_key.restype = ctypes.c_uint64
            L.orc_pair_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64]
            L.orc_pair_uniform.restype = ctypes.c_double
            L.orc_cbrt.argtypes = [ctypes.c_double]
            L.orc_cbrt.restype = ctypes.c_double
            L.orc_cbrtf.argtypes = [ctypes.c_float]
            L.orc_cbrtf.restype = ctypes.c_float
            L.orc_radius.argtypes = [ctypes.c_double]
            L.orc_radius.restype = ctypes.c_double
            L.orc_vt.argtypes = [_P(Params), ctypes.c_double]
            L.orc_vt.restype = ctypes.c_double
            L.orc_kernel.argtypes = [_P(Params), ctypes.c_double, ctypes.c_double]
            L.orc_kernel.restype = ctypes.c_double
            L.orc_kernelf.argtypes = [_P(Params), ctypes.c_float, ctypes.c_float]
            L.orc_kernelf.restype = ctypes.c_float
            L.orc_efficiency_long.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_efficiency_long.restype = ctypes.c_double
            L.orc_efficiency_longf.argtypes = [ctypes.c_float, ctypes.c_float]
            L.orc_efficiency_longf.restype = ctypes.c_float
            L.orc_scale.argtypes = [_P(Params), ctypes.c_int64]
            L.orc_scale.restype = ctypes.c_double
            L.orc_probability.argtypes = [_P(Params), ctypes.c_double, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
            L.orc_probability.restype = ctypes.c_double
            L.orc_gamma.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64]
            L.orc_gamma.restype = ctypes.c_int64
            L.orc_update.argtypes = [ctypes.c_int64, _i64p, _i64p, _f64p, _f64p]
            L.orc_update.restype = None
            L.orc_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, _i64p, ctypes.c_int64, _i64p]
            L.orc_permutation.restype = ctypes.c_int64
            L.orc_order.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
            L.orc_order.restype = ctypes.c_int
            L.orc_step.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                   _i64p, _f64p, ctypes.c_int64, _P(Stats)]
            L.orc_step.restype = ctypes.c_int
            L.orc_run.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                  _i64p, _f64p, ctypes.c_int64, ctypes.c_int64, _P(Stats)]
            L.orc_run.restype = ctypes.c_int
            L.orc_spectrum.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                       _i64p, _f64p, _f64p, ctypes.c_int32, ctypes.c_int32, _f64p]
            L.orc_spectrum.restype = ctypes.c_int
            L.orc_fall.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _f64p]
            L.orc_fall.restype = ctypes.c_int32
            L.orc_fall_distance.argtypes = [_P(Params), ctypes.c_double]
            L.orc_fall_distance.restype = ctypes.c_double
            L.orc_sediment.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       _i64p, _f64p, _i32p, _f64p, _f64p]
            L.orc_sediment.restype = ctypes.c_int
            L.orc_condense.argtypes = [_P(Params), ctypes.c_int64, ctypes.c_int32, _i32p, _i64p, _f64p, _f64p, _f64p,
                                       ctypes.c_double, _f64p]
            L.orc_condense.restype = ctypes.c_int
            L.orc_zeta_of.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]
            L.orc_zeta_of.restype = ctypes.c_double
            L.orc_z_of.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]
            L.orc_z_of.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


# ------------------------------------------------------------------ primitives
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def sort_key(seed, rank, cell, s):
    return int(lib().orc_sort_key(seed, rank, cell, s))


def pair_uniform(seed, pair, cell, s):
    return float(lib().orc_pair_uniform(seed, pair, cell, s))


def cbrt(x):
    f = lib().orc_cbrt
    return np.array([f(float(t)) for t in np.ravel(x)], dtype=np.float64).reshape(np.shape(x))


def cbrtf(x):
    f = lib().orc_cbrtf
    return np.array([f(float(t)) for t in np.ravel(np.asarray(x, np.float32))], dtype=np.float32).reshape(np.shape(x))


def radius(v):
    return lib().orc_radius(float(v))


def vt(P, r):
    return lib().orc_vt(ctypes.byref(P), float(r))


def kernel(P, vj, vk):
    return lib().orc_kernel(ctypes.byref(P), float(vj), float(vk))


def kernelf(P, vj, vk):
    return lib().orc_kernelf(ctypes.byref(P), float(vj), float(vk))


def efficiency_long(rj, rk):
    return lib().orc_efficiency_long(float(rj), float(rk))


def efficiency_longf(rj, rk):
    return lib().orc_efficiency_longf(float(rj), float(rk))


def scale(P, n_c):
    return lib().orc_scale(ctypes.byref(P), int(n_c))


def probability(P, scale_c, xi_j, vj, vk):
    return lib().orc_probability(ctypes.byref(P), float(scale_c), int(xi_j), float(vj), float(vk))


def gamma(p, u, xi_j, xi_k):
    return int(lib().orc_gamma(float(p), float(u), int(xi_j), int(xi_k)))


def update(g, xi_j, xi_k, vj, vk):
    a = (ctypes.c_int64(xi_j), ctypes.c_int64(xi_k), ctypes.c_double(vj), ctypes.c_double(vk))
    lib().orc_update(int(g), ctypes.byref(a[0]), ctypes.byref(a[1]), ctypes.byref(a[2]), ctypes.byref(a[3]))
    return a[0].value, a[1].value, a[2].value, a[3].value


def order(key_a, rank_a, key_b, rank_b):
    return int(lib().orc_order(key_a, rank_a, key_b, rank_b))


def permutation(seed, cell, s, xi_members):
    xm = np.ascontiguousarray(xi_members, dtype=np.int64)
    perm = np.zeros(max(len(xm), 1), dtype=np.int64)
    n_c = lib().orc_permutation(seed, cell, s, _ptr(xm, ctypes.c_int64), len(xm), _ptr(perm, ctypes.c_int64))
    if n_c < 0:
        raise MemoryError("oracle permutation")
    return perm[:n_c].copy()


# ------------------------------------------------------------------ full state
@dataclass
class State:
    """SD attributes indexed by SD id."""

    xi: np.ndarray  # int64 multiplicity
    v: np.ndarray  # float64 volume, m^3
    cell: np.ndarray  # int32 cell within the instance
    inst: np.ndarray | None  # int32 instance, or None
    n_cells: int
    n_inst: int = 1

    def copy(self) -> "State":
        return State(self.xi.copy(), self.v.copy(), self.cell.copy(),
                     None if self.inst is None else self.inst.copy(), self.n_cells, self.n_inst)

    def _args(self):
        self.xi = np.ascontiguousarray(self.xi, dtype=np.int64)
        self.v = np.ascontiguousarray(self.v, dtype=np.float64)
        self.cell = np.ascontiguousarray(self.cell, dtype=np.int32)
        if self.inst is not None:
            self.inst = np.ascontiguousarray(self.inst, dtype=np.int32)
        return (len(self.xi), self.n_cells, self.n_inst, _ptr(self.cell, ctypes.c_int32),
                _ptr(self.inst, ctypes.c_int32), _ptr(self.xi, ctypes.c_int64), _ptr(self.v, ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def step(P: Params, st: State, s: int) -> Stats:
    """One step with index s, in place."""
    stats = Stats()
    _check(lib().orc_step(ctypes.byref(P), *st._args(), int(s), ctypes.byref(stats)), "step")
    return stats


def run(P: Params, st: State, s0: int, n_steps: int) -> Stats:
    """Steps s0 .. s0 + n_steps - 1, in place."""
    stats = Stats()
    _check(lib().orc_run(ctypes.byref(P), *st._args(), int(s0), int(n_steps), ctypes.byref(stats)), "run")
    return stats


def spectrum(P: Params, st: State, edges, per_cell=False) -> np.ndarray:
    """dv/dlnr per radius bin (m^3 of particles per m^3 of air per unit ln r)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(e) - 1
    n_out = st.n_cells * st.n_inst * nb if per_cell else nb
    out = np.zeros(n_out, dtype=np.float64)
    n, nc, ni, cp, ip, xp, vp = st._args()
    _check(lib().orc_spectrum(ctypes.byref(P), n, nc, ni, cp, ip, xp, vp, _ptr(e, ctypes.c_double),
                              len(e), int(bool(per_cell)), _ptr(out, ctypes.c_double)), "spectrum")
    return out.reshape(st.n_cells * st.n_inst, nb) if per_cell else out


# -------------------------------------------------------------- sedimentation
def fall(zeta, iz, d, dz):
    """(new level or -1, new zeta) of one SD falling d in one step."""
    out = ctypes.c_double()
    lvl = lib().orc_fall(float(zeta), int(iz), float(d), float(dz), ctypes.byref(out))
    return int(lvl), out.value


def fall_distance(P: Params, v):
    return lib().orc_fall_distance(ctypes.byref(P), float(v))


def zeta_of(z, cell, nx, dz):
    """Heights above the cells' bottoms from heights above the domain bottom."""
    f = lib().orc_zeta_of
    return np.array([f(float(a), int(c), int(nx), float(dz)) for a, c in zip(np.ravel(z), np.ravel(cell))])


def z_of(zeta, cell, nx, dz):
    f = lib().orc_z_of
    return np.array([f(float(a), int(c), int(nx), float(dz)) for a, c in zip(np.ravel(zeta), np.ravel(cell))])


def sediment(P: Params, st: State, nx: int, dz: float, zeta: np.ndarray) -> float:
    """One sedimentation step in place (st.cell and zeta); returns the
    precipitated volume sum(xi v) of the SDs that fell through the bottom."""
    if st.inst is not None:
        raise ValueError("sedimentation of a single instance only")
    n, nc, ni, cp, ip, xp, vp = st._args()
    if zeta.dtype != np.float64 or not zeta.flags.c_contiguous or len(zeta) != n:
        raise ValueError("zeta must be a contiguous float64 array of n_sd heights")
    pr = ctypes.c_double(0.0)
    _check(lib().orc_sediment(ctypes.byref(P), n, int(nx), nc, float(dz), xp, vp, cp,
                              _ptr(zeta, ctypes.c_double), ctypes.byref(pr)), "sediment")
    return pr.value


# --------------------------------------------------------------- condensation
def condense(P: Params, st: State, G, s, r_min: float, want_condensed: bool = True):
    """One condensation step in place (st.v); per-cell growth coefficient G
    (m^2 s^-1) and supersaturation s; returns sum(xi dV) per cell (m^3) or
    None."""
    if st.inst is not None:
        raise ValueError("condensation of a single instance only")
    n, nc, ni, cp, ip, xp, vp = st._args()
    Ga = np.ascontiguousarray(G, dtype=np.float64)
    sa = np.ascontiguousarray(s, dtype=np.float64)
    if len(Ga) != nc or len(sa) != nc:
        raise ValueError("G and s need one value per cell")
    out = np.zeros(nc, dtype=np.float64) if want_condensed else None
    _check(lib().orc_condense(ctypes.byref(P), n, nc, cp, xp, vp, _ptr(Ga, ctypes.c_double),
                              _ptr(sa, ctypes.c_double), float(r_min), _ptr(out, ctypes.c_double)), "condense")
    return out
