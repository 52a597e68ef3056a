"""The C ABI without a GPU: the library builds and loads, exports every
function include/sdm.h declares, and its host-only calls behave."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_17238_gb300 import build as B
    from paper_2103_17238_gb300 import sdm

    B.build()
    return sdm.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sdm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(sdm_[a-z_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported(lib):
    from paper_2103_17238_gb300 import sdm

    names = _declared()
    assert "sdm_create" in names and "sdm_coalescence_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(sdm.EXPORTS)


def test_config_default_is_the_paper_example(lib):
    from paper_2103_17238_gb300 import sdm

    c = sdm.sdm_config_default()
    assert (c.kernel, c.precision, c.golovin_b, c.dt, c.dv, c.n_cells) == (0, 0, 1500.0, 1.0, 1e6, 1)
    assert (c.ry_k1, c.ry_k2, c.ry_k3, c.ry_r1, c.ry_r2) == (1.19e8, 8e3, 201.0, 40e-6, 600e-6)


def test_ctypes_layout_matches_the_header(tmp_path):
    """Field offsets of the Python structures equal the C compiler's."""
    from paper_2103_17238_gb300 import sdm

    prog = ['#include <stdio.h>', '#include <stddef.h>', '#include "sdm.h"', 'int main(void){']
    for st in (sdm.sdm_config, sdm.sdm_info, sdm.sdm_tuning, sdm.sdm_diag):
        name = st.__name__
        prog.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            prog.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    prog.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for st in (sdm.sdm_config, sdm.sdm_info, sdm.sdm_tuning, sdm.sdm_diag):
        assert int(out[st.__name__]) == ctypes.sizeof(st)
        for f, _ in st._fields_:
            assert int(out[f"{st.__name__}.{f}"]) == getattr(st, f).offset, f


@pytest.mark.parametrize("field,value", [("dt", 0.0), ("dv", -1.0), ("kernel", 7), ("precision", 3),
                                         ("n_cells", 0), ("ry_r2", 1e-6), ("golovin_b", float("nan"))])
def test_create_rejects_bad_config_before_touching_the_gpu(lib, field, value):
    from paper_2103_17238_gb300 import sdm

    c = sdm.sdm_config_default()
    setattr(c, field, value)
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_create(c, 16, 0)
    assert e.value.status == sdm.SDM_EINVAL
    assert lib.sdm_last_error(None)


def test_destroy_null_and_footprint(lib):
    from paper_2103_17238_gb300 import sdm

    assert lib.sdm_destroy(None) == sdm.SDM_OK
    assert lib.sdm_batch_destroy(None) == sdm.SDM_OK
    small = sdm.sdm_footprint_bytes(4096, 1, 4096)
    assert small == (4096 + 1) * 20 + 2 * 4 + sdm.sdm_footprint_bytes(0, 1, 0) - (1 * 20 + 2 * 4)
    big = sdm.sdm_footprint_bytes(2**20, 1, 2**20)
    assert big > 2**20 * 20 + 2**20 * 8  # state, then rank and perm per SD of a big cell


def test_fuse_default_matches_the_header():
    import re

    from paper_2103_17238_gb300 import sdm

    txt = open(os.path.join(ROOT, "include", "sdm.h")).read()
    m = re.search(r"#define SDM_FUSE_STEPS_DEFAULT (\d+)", txt)
    assert m and int(m.group(1)) == sdm.FUSE_STEPS_DEFAULT


def test_tuning_round_trip_and_validation(lib):
    """The launch tuning is host state: set, read back, rejected when out of
    range (the previous setting stays), restored by NULL."""
    from paper_2103_17238_gb300 import sdm

    default = {"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2,
               "fuse_steps": sdm.FUSE_STEPS_DEFAULT, "mid_max_sd": sdm.MID_MAX_SD_DEFAULT}
    sdm.sdm_set_tuning(None)
    assert sdm.sdm_get_tuning() == default
    t = {"smem_max_sd": 1024, "warp_cell_max": 128, "warps_per_block": 4, "fuse_steps": sdm.FUSE_STEPS_DEFAULT,
         "mid_max_sd": sdm.MID_MAX_SD_DEFAULT}
    sdm.sdm_set_tuning({k: t[k] for k in ("smem_max_sd", "warp_cell_max", "warps_per_block")})
    assert sdm.sdm_get_tuning() == t
    t = {"smem_max_sd": 1024, "warp_cell_max": 128, "warps_per_block": 4, "fuse_steps": 1024, "mid_max_sd": 0}
    sdm.sdm_set_tuning(t)
    assert sdm.sdm_get_tuning() == t
    t = {"smem_max_sd": 1024, "warp_cell_max": 128, "warps_per_block": 4, "fuse_steps": 0, "mid_max_sd": 20000}
    sdm.sdm_set_tuning(t)
    assert sdm.sdm_get_tuning() == t
    for bad in ({"smem_max_sd": 8192, "warp_cell_max": 256, "warps_per_block": 2},
                {"smem_max_sd": 1000, "warp_cell_max": 256, "warps_per_block": 2},
                {"smem_max_sd": 4096, "warp_cell_max": 1024, "warps_per_block": 2},
                {"smem_max_sd": 512, "warp_cell_max": 1024, "warps_per_block": 2},
                {"smem_max_sd": 4096, "warp_cell_max": 96, "warps_per_block": 2},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 3},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 0},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 2, "fuse_steps": 1025},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 2, "mid_max_sd": 70000},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 2, "mid_max_sd": 2048},
                {"smem_max_sd": 4096, "warp_cell_max": 256, "warps_per_block": 2, "fuse_steps": -1}):
        with pytest.raises(sdm.SdmError) as e:
            sdm.sdm_set_tuning(bad)
        assert e.value.status == sdm.SDM_EINVAL
        assert sdm.sdm_get_tuning() == t
    raw = sdm.sdm_tuning(4096, 256, 2, 2000)  # beyond the fusion limit
    assert lib.sdm_set_tuning(ctypes.byref(raw)) == sdm.SDM_EINVAL
    assert lib.sdm_get_tuning(None) == sdm.SDM_EINVAL
    # cells above the shared-memory threshold need multi-pass scratch
    assert sdm.sdm_footprint_bytes(4096, 1, 2048) > sdm.sdm_footprint_bytes(4096, 1, 1024)
    sdm.sdm_set_tuning(None)
    assert sdm.sdm_footprint_bytes(4096, 1, 2048) == sdm.sdm_footprint_bytes(4096, 1, 1024)


def test_autotune_candidates_are_valid_and_signature_is_stable(lib):
    from paper_2103_17238_gb300 import autotune, sdm

    seen = set()
    for c in autotune.CANDIDATES:
        sdm.sdm_set_tuning(c)
        seen.add(tuple(sorted(c.items())))
    sdm.sdm_set_tuning(None)
    assert len(seen) == len(autotune.CANDIDATES)
    assert {"smem_max_sd": 4096, "warp_cell_max": 512, "warps_per_block": 2} in autotune.CANDIDATES

    class FakeRun:
        def __init__(self, kernel, n_cells, largest):
            self.cfg = sdm.make_config(kernel, "fp64", n_cells=n_cells)
            self._info = sdm.sdm_info(n_sd=n_cells * largest, capacity_sd=n_cells * largest, step=0,
                                      device_bytes=0, n_cells=n_cells, largest_cell=largest)

        def info(self):
            return self._info

    a = autotune.signature([FakeRun("golovin", 1000, 200), FakeRun("geometric", 64, 3000)])
    b = autotune.signature([FakeRun("golovin", 1100, 250), FakeRun("geometric", 60, 2900)])
    c = autotune.signature([FakeRun("golovin", 1000, 600)])
    assert a == b and a != c


def test_selftest_rejects_bad_poll_counts_before_touching_the_gpu(lib):
    from paper_2103_17238_gb300 import sdm

    for polls in (0, -5, (1 << 24) + 1):
        assert sdm.sdm_selftest_bounded_wait(polls) == sdm.SDM_EINVAL
        assert b"max_polls" in lib.sdm_last_error(None)


def test_diagnostics_rejects_null_context(lib):
    from paper_2103_17238_gb300 import sdm

    d = sdm.sdm_diag()
    assert lib.sdm_diagnostics(None, ctypes.byref(d)) == sdm.SDM_EINVAL
