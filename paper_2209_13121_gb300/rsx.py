"""Python binding of libprsoxs_gb300.so (the C ABI in include/rsx.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  torch tensors supply device memory and streams.  Importing this
module loads the library and raises if it is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build_ext import lib_path

RSX_OK = 0
RSX_ERR_INVALID = -1
RSX_ERR_OOM = -2
RSX_ERR_CUDA = -3
RSX_ERR_UNSUPPORTED = -4
RSX_ERR_STATE = -5
RSX_HOST = 0
RSX_DEVICE = 1
RSX_HOST_ASYNC = 2
RSX_FRAME_LITERAL = 0
RSX_FRAME_LAB = 1
RSX_MAX_COMPONENTS = 32

EXPORTED = (
    "rsx_create", "rsx_destroy", "rsx_last_error", "rsx_workspace_bytes", "rsx_angle_count",
    "rsx_set_morphology", "rsx_set_optical_constants", "rsx_run", "rsx_polarization",
    "rsx_fft3d", "rsx_ewald", "rsx_rotate_accumulate", "rsx_scatter_angle",
    "rsx_set_timing", "rsx_phase_times", "rsx_scatter_angle_noalloc", "rsx_nt",
    "rsx_set_wait_limit", "rsx_check", "rsx_angle_batch", "rsx_zfirst_plan",
    "rsx_zfirst_plan_for",
)
MAX_ANGLE_BATCH = 8
NOALLOC_MAX_VOXELS = 1 << 20
NOALLOC_MAX_PIXELS = 1 << 16
PHASES = ("pol_fftx", "ffty", "ewald", "rotate", "other", "nt", "fftx")


class RsxConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("n_components", ctypes.c_int),
        ("voxel_nm", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("algorithm", ctypes.c_int),
        ("frame", ctypes.c_int),
        ("validate", ctypes.c_int),
        ("angle_batch", ctypes.c_int),
    ]


class RsxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rsx error {code}: {msg}")
        self.code = code


def load_library(path: str | None = None) -> ctypes.CDLL:
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2209_13121_gb300.build_ext first "
                           "(the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "rsx_create": (ci, [ctypes.POINTER(RsxConfig), ctypes.POINTER(vp)]),
        "rsx_destroy": (ci, [vp]),
        "rsx_last_error": (ctypes.c_char_p, []),
        "rsx_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(RsxConfig)]),
        "rsx_angle_count": (ci, [cd, cd, cd, ci]),
        "rsx_set_morphology": (ci, [vp, vp, ci, vp]),
        "rsx_set_optical_constants": (ci, [vp, ci, vp, vp]),
        "rsx_run": (ci, [vp, cd, cd, cd, ci, vp, ci, vp, ci, vp]),
        "rsx_polarization": (ci, [vp, ci, cd, vp, vp]),
        "rsx_fft3d": (ci, [vp, vp, vp]),
        "rsx_ewald": (ci, [vp, ci, vp, vp, vp]),
        "rsx_rotate_accumulate": (ci, [vp, vp, cd, vp, vp]),
        "rsx_scatter_angle": (ci, [vp, ci, cd, vp, vp]),
        "rsx_set_timing": (ci, [vp, ci]),
        "rsx_set_wait_limit": (ci, [vp, ctypes.c_longlong]),
        "rsx_phase_times": (ci, [vp, vp, vp]),
        "rsx_scatter_angle_noalloc": (ci, [vp, ci, ci, ci, ci, cd, cd, vp, cd, ci, vp, vp]),
        "rsx_nt": (ci, [vp, ci, vp, vp]),
        "rsx_check": (ci, [vp, vp]),
        "rsx_angle_batch": (ci, [vp]),
        "rsx_zfirst_plan": (ci, [vp, ci, vp, vp, vp]),
        "rsx_zfirst_plan_for": (ci, [ctypes.POINTER(RsxConfig), cd, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(rc):
    if rc != RSX_OK:
        raise RsxError(rc, lib().rsx_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def angle_count(start, inc, end, rotation=True) -> int:
    return lib().rsx_angle_count(start, inc, end, 1 if rotation else 0)


def _device_buffer(t, what, dtype_name, shape=None, numel=None, device=None):
    """Address of a torch CUDA tensor the library will read or write, after
    checking that it is one: on a CUDA device (the context's, when given),
    of the context's real type, contiguous and of the expected size.  The
    library borrows the address unchecked beyond that, so a wrong buffer
    would be read or written out of bounds on the GPU."""
    if isinstance(t, int):
        return ctypes.c_void_p(t)  # a raw device address: the caller vouches for it
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, the context on cuda:{device}")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"{what} must be {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def make_config(nx, ny, nz, n_components, voxel_nm, precision=32, algorithm=1,
                frame=RSX_FRAME_LITERAL, validate=False, angle_batch=0) -> RsxConfig:
    return RsxConfig(nx, ny, nz, n_components, voxel_nm, precision, algorithm, frame,
                     1 if validate else 0, angle_batch)


def workspace_bytes(cfg: RsxConfig) -> int:
    return lib().rsx_workspace_bytes(ctypes.byref(cfg))


def zfirst_plan_for(cfg: RsxConfig, energy_ev) -> tuple:
    """rsx_zfirst_plan_for: (n_planes, first_bin, angles_per_pass) of the
    z-first path for a context of this configuration at this energy (host
    only, no GPU needed); n_planes = 0 when the path does not serve it."""
    ns, kb, kz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().rsx_zfirst_plan_for(ctypes.byref(cfg), float(energy_ev), ctypes.byref(ns),
                                     ctypes.byref(kb), ctypes.byref(kz)))
    return ns.value, kb.value, kz.value


class Context:
    """One simulation context (a grid, a material count and a precision).

    Device buffers passed to the methods are torch CUDA tensors (or raw
    integer addresses); host buffers are numpy arrays."""

    def __init__(self, nx, ny, nz, n_components, voxel_nm, precision=32, algorithm=1,
                 frame=RSX_FRAME_LITERAL, validate=False, angle_batch=0):
        self.cfg = make_config(nx, ny, nz, n_components, voxel_nm, precision, algorithm,
                               frame, validate, angle_batch)
        self.real = np.float32 if precision == 32 else np.float64
        self._dt = "float32" if precision == 32 else "float64"
        h = ctypes.c_void_p()
        _check(lib().rsx_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self._h = h
        import torch
        self.device = torch.cuda.current_device()
        self._keep = None  # keeps a borrowed device morphology alive

    @property
    def angle_batch(self):
        """e-field angles per read of the morphology in rsx_run (Algorithm 1)."""
        return lib().rsx_angle_batch(self._h)

    def zfirst_plan(self, energy_index):
        """(n_planes, first_bin, angles_per_pass) of the z-first path for this
        energy (rsx_zfirst_plan); n_planes = 0 when the path does not serve it."""
        ns, kb, kz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().rsx_zfirst_plan(self._h, int(energy_index), ctypes.byref(ns),
                                     ctypes.byref(kb), ctypes.byref(kz)))
        return ns.value, kb.value, kz.value

    @property
    def shape(self):
        return (self.cfg.nz, self.cfg.ny, self.cfg.nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().rsx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ inputs
    def set_morphology(self, M, stream=None, async_copy=False):
        """M: [c][nz][ny][nx][4] (v, s, phi, theta).  numpy -> copied from
        host; torch CUDA tensor -> borrowed (kept alive by this object).
        async_copy (numpy in page-locked memory, e.g. a pinned torch
        tensor's .numpy()): the copy is only enqueued on `stream`; M must
        stay unchanged until the stream has passed it."""
        if isinstance(M, np.ndarray):
            A = np.ascontiguousarray(M, dtype=self.real)
            self._check_shape(A.shape)
            where = RSX_HOST_ASYNC if async_copy else RSX_HOST
            _check(lib().rsx_set_morphology(self._h, A.ctypes.data_as(ctypes.c_void_p), where,
                                            _stream_handle(stream) if stream is not None else None))
            if async_copy:
                self._keep = A
                return
            # Algorithm 2 streams from this host array on every energy
            self._keep = A if self.cfg.algorithm >= 2 else None
            return
        c = self.cfg
        ptr = _device_buffer(M, "device morphology", self._dt,
                             shape=(c.n_components, c.nz, c.ny, c.nx, 4), device=self.device)
        _check(lib().rsx_set_morphology(self._h, ptr, RSX_DEVICE, _stream_handle(stream)))
        self._keep = M

    def _check_shape(self, shp):
        want = (self.cfg.n_components, self.cfg.nz, self.cfg.ny, self.cfg.nx, 4)
        if tuple(shp) != want:
            raise ValueError(f"morphology shape {shp}, expected {want}")

    def set_optical_constants(self, energies, constants):
        E = np.ascontiguousarray(energies, dtype=np.float64)
        K = np.ascontiguousarray(constants, dtype=np.float64)
        if K.shape != (E.size, self.cfg.n_components, 4):
            raise ValueError(f"constants shape {K.shape}, expected {(E.size, self.cfg.n_components, 4)}")
        _check(lib().rsx_set_optical_constants(self._h, E.size, E.ctypes.data_as(ctypes.c_void_p),
                                               K.ctypes.data_as(ctypes.c_void_p)))
        self.n_energies = E.size

    # --------------------------------------------------------- simulation
    def run(self, angles=(0.0, 1.0, 0.0), rotation=True, energy_indices=None, out=None,
            stream=None):
        """Algorithm 1 for the selected energies.  out: None (returns a new
        host numpy array), a numpy array (host) or a torch CUDA tensor."""
        sel = None
        n_sel = getattr(self, "n_energies", 0)
        if energy_indices is not None:
            sel = np.ascontiguousarray(energy_indices, dtype=np.int32)
            n_sel = sel.size
        shape = (n_sel, self.cfg.ny, self.cfg.nx)
        if out is None:
            out = np.empty(shape, dtype=self.real)
        if isinstance(out, np.ndarray):
            if out.shape != shape or out.dtype != self.real or not out.flags.c_contiguous:
                raise ValueError("host output has the wrong shape, dtype or layout")
            ptr, where = out.ctypes.data_as(ctypes.c_void_p), RSX_HOST
            st = _stream_handle(stream) if stream is not None else None
        else:
            ptr = _device_buffer(out, "device output", self._dt, shape=shape, device=self.device)
            where = RSX_DEVICE
            st = _stream_handle(stream)
        _check(lib().rsx_run(self._h, float(angles[0]), float(angles[1]), float(angles[2]),
                             1 if rotation else 0,
                             sel.ctypes.data_as(ctypes.c_void_p) if sel is not None else None,
                             n_sel, ptr, where, st))
        return out

    def check(self, stream=None):
        """rsx_check: waits for `stream` and raises RsxError (RSX_ERR_CUDA)
        if a pipelined kernel of this context timed out since the last
        check; device results written since then are then not valid."""
        _check(lib().rsx_check(self._h, _stream_handle(stream)))

    # ------------------------------------------------------------ timing
    def set_timing(self, enable=True):
        _check(lib().rsx_set_timing(self._h, 1 if enable else 0))

    def set_wait_limit(self, polls=None):
        """Bound of the pipelined kernels' copy waits (None: the default);
        0 makes them run out at once, to exercise the failure path."""
        _check(lib().rsx_set_wait_limit(self._h, -1 if polls is None else int(polls)))

    def phase_times(self):
        """{phase: (total device ms, kernel launches)} since the last call."""
        ms = (ctypes.c_double * len(PHASES))()
        n = (ctypes.c_longlong * len(PHASES))()
        _check(lib().rsx_phase_times(self._h, ms, n))
        return {name: (ms[i], n[i]) for i, name in enumerate(PHASES)}

    # ------------------------------------------------------- single steps
    def _buf(self, t, what, numel):
        return _device_buffer(t, what, self._dt, numel=numel, device=self.device)

    def _n(self):
        return self.cfg.nx * self.cfg.ny * self.cfg.nz

    def _npix(self):
        return self.cfg.nx * self.cfg.ny

    def polarization(self, energy_index, alpha_rad, p_out, stream=None):
        """p_out: [3][nz][ny][nx][2] (complex as re, im pairs)."""
        ptr = self._buf(p_out, "p_out", 6 * self._n())
        _check(lib().rsx_polarization(self._h, int(energy_index), float(alpha_rad), ptr,
                                      _stream_handle(stream)))
        return p_out

    def nt(self, energy_index, nt_out, stream=None):
        """Algorithm 3's N_t (entries xx, xy, yy, xz, yz) into nt_out [5][nz][ny][nx][2]."""
        ptr = self._buf(nt_out, "nt_out", 10 * self._n())
        _check(lib().rsx_nt(self._h, int(energy_index), ptr, _stream_handle(stream)))
        return nt_out

    def fft3d(self, p, stream=None):
        ptr = self._buf(p, "p", 6 * self._n())
        _check(lib().rsx_fft3d(self._h, ptr, _stream_handle(stream)))
        return p

    def ewald(self, energy_index, p_tilde, img_out, stream=None):
        pt = self._buf(p_tilde, "p_tilde", 6 * self._n())
        im = self._buf(img_out, "img_out", self._npix())
        _check(lib().rsx_ewald(self._h, int(energy_index), pt, im, _stream_handle(stream)))
        return img_out

    def rotate_accumulate(self, img, alpha_rad, acc, stream=None):
        im = self._buf(img, "img", self._npix())
        ac = self._buf(acc, "acc", self._npix())
        _check(lib().rsx_rotate_accumulate(self._h, im, float(alpha_rad), ac,
                                           _stream_handle(stream)))
        return acc

    def scatter_angle(self, energy_index, alpha_rad, img_out, stream=None):
        im = self._buf(img_out, "img_out", self._npix())
        _check(lib().rsx_scatter_angle(self._h, int(energy_index), float(alpha_rad), im,
                                       _stream_handle(stream)))
        return img_out


def scatter_angle_noalloc(M, energy_ev, constants, alpha_rad, img_out, voxel_nm,
                          frame=RSX_FRAME_LITERAL, stream=None):
    """rsx_scatter_angle_noalloc: the unrotated FP32 detector image for one
    energy and angle, without any device allocation (fixed in-library
    scratch; see include/rsx.h for the size limits).  M: contiguous float32
    CUDA tensor [c][nz][ny][nx][4]; constants: [c][4]; img_out: float32 CUDA
    tensor [ny][nx]."""
    if len(M.shape) != 5 or M.shape[4] != 4:
        raise ValueError("M must be [c][nz][ny][nx][4]")
    c, nz, ny, nx, _ = M.shape
    mp = _device_buffer(M, "M", "float32")
    ip = _device_buffer(img_out, "img_out", "float32", shape=(ny, nx), device=M.device.index)
    K = np.ascontiguousarray(constants, dtype=np.float64).reshape(c, 4)
    _check(lib().rsx_scatter_angle_noalloc(
        mp, nx, ny, nz, c, float(voxel_nm), float(energy_ev),
        K.ctypes.data_as(ctypes.c_void_p), float(alpha_rad), int(frame), ip,
        _stream_handle(stream)))
    return img_out
