"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/rsx.h declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2209_13121_gb300 import build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build_ext.build()
    from paper_2209_13121_gb300 import rsx
    return rsx.load_library(path)


def _declared():
    txt = open(os.path.join(ROOT, "include", "rsx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rsx_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_binding_names():
    from paper_2209_13121_gb300 import rsx
    assert _declared() == sorted(rsx.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_angle_count_host_only(lib):
    from paper_2209_13121_gb300 import rsx
    assert rsx.angle_count(0, 2, 180) == 91
    assert rsx.angle_count(0, 30, 180) == 7
    assert rsx.angle_count(0, 7, 20) == 3
    assert rsx.angle_count(10, 5, 10) == 1
    assert rsx.angle_count(0, 2, 180, rotation=False) == 1
    assert rsx.angle_count(0, 0, 180) == -1
    assert rsx.angle_count(0, -1, 180) == -1
    assert rsx.angle_count(10, 1, 0) == -1
    assert rsx.angle_count(float("nan"), 1, 2) == -1


def test_workspace_bytes_follows_table1(lib):
    from paper_2209_13121_gb300 import rsx
    nx, ny, nz, c = 1024, 1024, 128, 4
    cfg = rsx.make_config(nx, ny, nz, c, 5.0, precision=32)
    N, npix = nx * ny * nz, nx * ny
    b = rsx.workspace_bytes(cfg)
    table1 = (4 * c + 6) * N * 4 + 2 * npix * 4   # (4c+6) N + 2 nx ny Real
    # beyond Table 1: per-pixel geometry (32 B) and, for FP32 grids the fused
    # y+z pass takes, the two q_z bins of three fields in up to four partial
    # slots (192 B)
    assert table1 <= b <= table1 + 224 * npix + 64 * (nx + ny + nz) + 64
    assert rsx.workspace_bytes(rsx.make_config(1000, 1024, 1, 2, 5.0)) == 0  # nx not 2^k
    assert rsx.workspace_bytes(rsx.make_config(8, 8, 1, 0, 5.0)) == 0        # c = 0
    assert rsx.workspace_bytes(rsx.make_config(8, 8, 1, 2, 5.0, precision=16)) == 0


def test_create_rejects_bad_config_before_touching_a_gpu(lib):
    from paper_2209_13121_gb300 import rsx
    h = ctypes.c_void_p()
    for cfg in (rsx.make_config(12, 8, 1, 2, 5.0), rsx.make_config(8, 8, 0, 2, 5.0),
                rsx.make_config(8, 8, 1, 33, 5.0), rsx.make_config(8, 8, 1, 2, -1.0),
                rsx.make_config(8, 8, 1, 2, 5.0, precision=16),
                rsx.make_config(8, 8, 1, 2, 5.0, frame=7)):
        rc = lib.rsx_create(ctypes.byref(cfg), ctypes.byref(h))
        assert rc == rsx.RSX_ERR_INVALID
        assert lib.rsx_last_error().decode()
    assert lib.rsx_destroy(None) == rsx.RSX_OK
