"""The z-first path's plan (rsx_zfirst_plan_for, host arithmetic only, no
GPU): for every shape the path serves, voxel sizes of 2, 5 and 10 nm and
energies from well below to well above the carbon edge, the run of q_z
planes it keeps holds both bins (b0 = floor(t) and b0 + 1 of Eq. (Ewald))
of every detector pixel on the sphere as the oracle's geometry computes
them, ends at bin 1, keeps no more than one bin beyond the lowest one read,
and fits the angle batch; shapes, precisions and algorithms the path does
not serve get no plan, and bad arguments are refused."""
import math

import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O
from paper_2209_13121_gb300 import build_ext

VOXEL = 5.0


@pytest.fixture(scope="module")
def rsx():
    build_ext.build()
    from paper_2209_13121_gb300 import rsx as R
    return R


def _bins_read(shape, E, dv=VOXEL):
    """The q_z bins b0 and b0 + 1 (mod nz) that the pixels on the Ewald
    sphere read, from the oracle's q grid and Eq. (Ewald), and the lowest
    b0 (unreduced)."""
    nz, ny, nx = shape
    k = O.wavenumber(E)
    qx = O.q_axis(nx, dv)[None, :]
    qy = O.q_axis(ny, dv)[:, None]
    rad = k * k - qx * qx - qy * qy
    on = rad >= 0.0
    t = (-k + np.sqrt(np.where(on, rad, 0.0))) / (2.0 * math.pi / (nz * dv))
    z0 = np.floor(t[on]).astype(np.int64)
    return set(np.mod(z0, nz).tolist()) | set(np.mod(z0 + 1, nz).tolist()), int(z0.min())


SHAPES = [(32, 512, 512), (64, 1024, 512), (128, 512, 1024), (128, 1024, 1024),
          (64, 2048, 2048), (32, 512, 2048), (128, 2048, 2048)]
ENERGIES = [150.0, 170.0, 200.0, 250.0, 270.0, 285.0, 300.0, 320.0, 400.0, 700.0]


@pytest.mark.parametrize("shape", SHAPES, ids=["x".join(map(str, s)) for s in SHAPES])
@pytest.mark.parametrize("batch", [0, 1, 3])
@pytest.mark.parametrize("dv", [VOXEL, 2.0, 10.0])
def test_plan_covers_every_bin_read(rsx, shape, batch, dv):
    nz, ny, nx = shape
    cfg = rsx.make_config(nx, ny, nz, 4, dv, angle_batch=batch)
    kx = batch if batch else min(8, max(1, int((32 << 30) / (3.0 * nx * ny * nz * 8))))
    served = 0
    for E in ENERGIES:
        ns, kb, kz = rsx.zfirst_plan_for(cfg, E)
        need, lowest = _bins_read(shape, E, dv)
        want_ns = 2 - lowest   # bins lowest .. 1 (one more below near a bin edge)
        if ns == 0:   # most bins read: the path steps aside
            assert kz == 0 and kb == 0 and 4 * (want_ns + 1) > 3 * nz, (E, want_ns)
            continue
        served += 1
        assert ns in (want_ns, want_ns + 1) and 4 * ns <= 3 * nz, (E, ns, want_ns)
        run = {(kb + s) % nz for s in range(ns)}
        assert need <= run, (E, sorted(need - run))
        assert (kb + ns - 1) % nz == 1   # the run ends at bin 1
        assert kz == min(32, kx * nz // ns) and kz * ns <= kx * nz
    assert served >= (5 if dv == VOXEL else 1)


def test_benchmark_plan(rsx):
    """1024 x 1024 x 128, 5 nm voxels, the default batch of 8: the planes the
    benchmark's energies keep (270 and 320 eV bound the 150) and the angles
    per morphology read."""
    cfg = rsx.make_config(1024, 1024, 128, 4, VOXEL)
    assert rsx.zfirst_plan_for(cfg, 270.0) == (36, 94, 28)
    assert rsx.zfirst_plan_for(cfg, 320.0) == (30, 100, 32)


def test_no_plan_where_the_path_does_not_serve(rsx):
    for (nz, ny, nx), prec, alg in (((16, 512, 512), 32, 1), ((32, 512, 512), 64, 1),
                                    ((32, 512, 512), 32, 2), ((32, 512, 512), 32, 3),
                                    ((32, 256, 512), 32, 1), ((256, 512, 512), 32, 1),
                                    ((128, 1024, 1000), 32, 1)):
        cfg = rsx.make_config(nx, ny, nz, 2, VOXEL, precision=prec, algorithm=alg)
        assert rsx.zfirst_plan_for(cfg, 285.0) == (0, 0, 0), ((nz, ny, nx), prec, alg)


def test_bad_arguments_are_refused(rsx):
    cfg = rsx.make_config(1024, 1024, 128, 4, VOXEL)
    for E in (0.0, -5.0, float("nan"), float("inf")):
        with pytest.raises(rsx.RsxError):
            rsx.zfirst_plan_for(cfg, E)
    with pytest.raises(rsx.RsxError):
        rsx.zfirst_plan_for(rsx.make_config(1024, 1024, 0, 4, VOXEL), 285.0)
