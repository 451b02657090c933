"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/rsx.h declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import numpy as np
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
    cfg = rsx.make_config(nx, ny, nz, c, 5.0, precision=32, angle_batch=1)
    N, npix = nx * ny * nz, nx * ny
    b = rsx.workspace_bytes(cfg)
    table1 = (4 * c + 6) * N * 4 + 2 * npix * 4   # (4c+6) N + 2 nx ny Real
    # beyond Table 1: per-pixel geometry (32 B) and, for FP32 grids the fused
    # y+z pass takes, the two q_z bins of three fields in up to four partial
    # slots (192 B) and each pixel's lower bin index (2 B)
    assert table1 <= b <= table1 + 226 * npix + 64 * (nx + ny + nz) + 64
    # each further angle of a batch holds one more p (3 N complex float)
    for k in (2, 4, 8):
        assert rsx.workspace_bytes(rsx.make_config(nx, ny, nz, c, 5.0, angle_batch=k)) == \
            b + (k - 1) * 3 * N * 8
    # the default batch, and no batch where the multi-angle pass does not apply
    assert rsx.workspace_bytes(rsx.make_config(nx, ny, nz, c, 5.0)) == b + 7 * 3 * N * 8
    # nx = 2048 takes at most 3 on the multi-angle x pass (nz = 16), up to 8
    # where the z-first path serves the shape (nz = 32, 64, 128); other row
    # lengths none
    one = rsx.make_config(2048, 2048, 16, c, 5.0, angle_batch=1)
    assert rsx.workspace_bytes(rsx.make_config(2048, 2048, 16, c, 5.0, angle_batch=4)) == \
        rsx.workspace_bytes(one) + 2 * 3 * 2048 * 2048 * 16 * 8
    one = rsx.make_config(2048, 2048, 64, c, 5.0, angle_batch=1)
    assert rsx.workspace_bytes(rsx.make_config(2048, 2048, 64, c, 5.0, angle_batch=4)) == \
        rsx.workspace_bytes(one) + 3 * 3 * 2048 * 2048 * 64 * 8
    one = rsx.make_config(1000, 1024, 100, c, 5.0, angle_batch=1)
    assert rsx.workspace_bytes(rsx.make_config(1000, 1024, 100, c, 5.0, angle_batch=4)) == \
        rsx.workspace_bytes(one)
    assert rsx.workspace_bytes(rsx.make_config(nx, ny, nz, c, 5.0, precision=64, angle_batch=4)) \
        == rsx.workspace_bytes(rsx.make_config(nx, ny, nz, c, 5.0, precision=64, angle_batch=1))
    assert rsx.workspace_bytes(rsx.make_config(8, 8, 1, 2, 5.0, angle_batch=9)) == 0
    assert rsx.workspace_bytes(rsx.make_config(1000, 1024, 1, 2, 5.0)) > 0   # any nx <= 4096
    assert rsx.workspace_bytes(rsx.make_config(4097, 1024, 1, 2, 5.0)) == 0
    assert rsx.workspace_bytes(rsx.make_config(8, 0, 1, 2, 5.0)) == 0
    assert rsx.workspace_bytes(rsx.make_config(8, 8, 1, 0, 5.0)) == 0        # c = 0
    assert rsx.workspace_bytes(rsx.make_config(8, 8, 1, 2, 5.0, precision=16)) == 0


def test_create_rejects_bad_config_before_touching_a_gpu(lib):
    from paper_2209_13121_gb300 import rsx
    h = ctypes.c_void_p()
    for cfg in (rsx.make_config(4097, 8, 1, 2, 5.0), rsx.make_config(8, 0, 1, 2, 5.0),
                rsx.make_config(8, 8, 0, 2, 5.0), rsx.make_config(8, 8, 1, 2, 5.0, angle_batch=-1),
                rsx.make_config(8, 8, 1, 33, 5.0), rsx.make_config(8, 8, 1, 2, -1.0),
                rsx.make_config(8, 8, 1, 2, 5.0, precision=16),
                rsx.make_config(8, 8, 1, 2, 5.0, frame=7)):
        rc = lib.rsx_create(ctypes.byref(cfg), ctypes.byref(h))
        assert rc == rsx.RSX_ERR_INVALID
        assert lib.rsx_last_error().decode()
    assert lib.rsx_destroy(None) == rsx.RSX_OK


class _FakeTensor:
    """Stands in for a torch tensor in the binding's argument checks (no GPU
    needed): only the attributes those checks read."""

    def __init__(self, shape, dtype="torch.float32", is_cuda=True, contiguous=True, index=0):
        import types
        self.shape = shape
        self.dtype = dtype
        self.is_cuda = is_cuda
        self.device = types.SimpleNamespace(index=index)
        self._contig = contiguous

    def is_contiguous(self):
        return self._contig

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def data_ptr(self):
        return 4096


@pytest.mark.parametrize("bad,msg", [
    (dict(is_cuda=False), "CUDA tensor"),
    (dict(dtype="torch.float64"), "must be float32"),
    (dict(dtype="torch.float16"), "must be float32"),
    (dict(contiguous=False), "contiguous"),
    (dict(shape=(3, 5)), "shape"),
    (dict(index=1), "cuda:1"),
])
def test_binding_refuses_wrong_device_buffers(lib, bad, msg):
    from paper_2209_13121_gb300 import rsx
    kw = dict(shape=(4, 5))
    kw.update(bad)
    with pytest.raises(ValueError, match=msg):
        rsx._device_buffer(_FakeTensor(**kw), "img_out", "float32", shape=(4, 5), device=0)
    # the same buffer with every property right passes
    assert rsx._device_buffer(_FakeTensor((4, 5)), "img_out", "float32", shape=(4, 5),
                              device=0).value == 4096


def test_binding_refuses_element_count(lib):
    from paper_2209_13121_gb300 import rsx
    with pytest.raises(ValueError, match="elements"):
        rsx._device_buffer(_FakeTensor((3, 2, 8, 8, 2)), "p_out", "float32", numel=6 * 129)


def test_noalloc_refuses_host_tensors_in_the_binding(lib):
    torch = pytest.importorskip("torch")
    from paper_2209_13121_gb300 import rsx
    M = torch.zeros((1, 2, 8, 8, 4))
    out = torch.zeros((8, 8))
    with pytest.raises(ValueError, match="CUDA tensor"):
        rsx.scatter_angle_noalloc(M, 285.0, np.zeros((1, 4)), 0.0, out, 5.0)


def test_noalloc_refuses_host_pointers_in_the_c_abi(lib):
    """M and img_out must be device memory: host addresses are refused before
    any work is enqueued (no GPU is needed to see it)."""
    from paper_2209_13121_gb300 import rsx
    M = np.zeros((1, 2, 8, 8, 4), np.float32)
    out = np.zeros((8, 8), np.float32)
    K = np.zeros((1, 4))
    rc = lib.rsx_scatter_angle_noalloc(M.ctypes.data, 8, 8, 2, 1, 5.0, 285.0, K.ctypes.data, 0.0,
                                       0, out.ctypes.data, None)
    assert rc == rsx.RSX_ERR_INVALID
    assert "device" in lib.rsx_last_error().decode()


def test_check_needs_a_context(lib):
    from paper_2209_13121_gb300 import rsx
    assert lib.rsx_check(None, None) == rsx.RSX_ERR_INVALID
