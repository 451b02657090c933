"""The z-first path of Algorithm 1 (FP32, nz = 32, 64, 128; nx, ny = 512,
1024, 2048): p's z transform first, only the run of q_z bins the detector
pixels read kept, then the x and y transforms on those planes.  The 3-D DFT
is separable, so the result is Algorithm 1's up to rounding order: checked
against the oracle densely on one grid and at sampled output pixels (sparse
morphologies, exact by linearity of the DFT) on every kernel shape, in both
frames, with partial angle batches; plus the plan itself against the bins
the oracle's geometry reads, the energies where the path steps aside, and
bitwise independence from the angle batch."""
import math

import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O
from paper_2209_13121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VOXEL = 5.0


@pytest.fixture(scope="module")
def rsx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx as R
    return R


def _bins_read(shape, E):
    """The q_z bins b0 and b0 + 1 (mod nz) of every pixel on the sphere, from
    the oracle's geometry (Eq. (Ewald)), and the lowest b0 (unreduced)."""
    nz, ny, nx = shape
    k = O.wavenumber(E)
    qx = O.q_axis(nx, VOXEL)[None, :]
    qy = O.q_axis(ny, VOXEL)[:, None]
    rad = k * k - qx * qx - qy * qy
    on = rad >= 0.0
    t = (-k + np.sqrt(np.where(on, rad, 0.0))) / (2.0 * math.pi / (nz * VOXEL))
    z0 = np.floor(t[on]).astype(np.int64)
    return set(np.mod(z0, nz).tolist()) | set(np.mod(z0 + 1, nz).tolist()), int(z0.min())


def _sampled_check(got, ref, oy, ox, ny, nx):
    center = np.hypot(oy - ny // 2, ox - nx // 2) < 2.5
    np.testing.assert_allclose(got[center], ref[center], rtol=1e-5)
    rest = ~center
    rel = np.linalg.norm(got[rest] - ref[rest]) / np.linalg.norm(ref[rest])
    assert rel < 1e-4, rel
    big = rest & (ref > 1e-4 * ref[rest].max())
    assert big.sum() > 20
    assert (np.abs(got - ref)[big] / ref[big]).max() < 2e-3


PLAN = [(32, 512, 512), (64, 1024, 512), (128, 512, 1024), (128, 1024, 1024), (64, 2048, 2048),
        (32, 512, 2048)]


@pytest.mark.parametrize("shape", PLAN, ids=["x".join(map(str, s)) for s in PLAN])
def test_plan_covers_the_bins_every_pixel_reads(rsx, shape):
    nz, ny, nx = shape
    energies = [170.0, 175.0, 200.0, 270.0, 285.0, 310.0, 400.0]
    K = synth.optical_constants(energies, 2, seed=5)
    with rsx.Context(nx, ny, nz, 2, VOXEL, precision=32, angle_batch=1) as ctx:
        ctx.set_optical_constants(energies, K)
        kx = ctx.angle_batch
        for ie, E in enumerate(energies):
            ns, kb, kz = ctx.zfirst_plan(ie)
            need, lowest = _bins_read(shape, E)
            want_ns = 2 - lowest   # bins lowest .. 1 (one more below near a bin edge)
            if ns == 0:   # most bins read: the path steps aside
                assert kz == 0 and 4 * (want_ns + 1) > 3 * nz, (E, want_ns)
                continue
            assert ns in (want_ns, want_ns + 1) and 4 * ns <= 3 * nz, (E, ns, want_ns)
            run = {(kb + s) % nz for s in range(ns)}
            assert need <= run, (E, sorted(need - run))
            assert (kb + ns - 1) % nz == 1   # the run ends at bin 1
            assert kz == min(32, kx * nz // ns)
    # shapes and precisions the path does not serve
    for (nz, ny, nx), prec, alg in (((16, 512, 512), 32, 1), ((32, 512, 512), 64, 1),
                                    ((32, 512, 512), 32, 2), ((32, 256, 512), 32, 1),
                                    ((256, 512, 512), 32, 1)):
        with rsx.Context(nx, ny, nz, 2, VOXEL, precision=prec, algorithm=alg,
                         angle_batch=1) as ctx:
            ctx.set_optical_constants([285.0], synth.optical_constants([285.0], 2, seed=6))
            assert ctx.zfirst_plan(0) == (0, 0, 0)
    with rsx.Context(512, 512, 32, 2, VOXEL, precision=32, angle_batch=1) as ctx:
        with pytest.raises(rsx.RsxError):
            ctx.zfirst_plan(0)   # no optical constants yet


def test_dense_grid_matches_oracle(rsx):
    """32 x 512 x 512, c = 2 (nz = 32: one 32-point DFT per lane, 32-pixel
    tiles; the 512-row selection pass), four angles in two passes of 2
    (angle_batch 1: 32 // 10 angles per pass at most), against the dense
    FP64 oracle; device and host output identical."""
    shape, c, E = (32, 512, 512), 2, 285.0
    nz, ny, nx = shape
    M = synth.morphology_random(shape, c, seed=41, dtype=np.float32)
    K = synth.optical_constants([E], c, seed=42)
    angles = (0.0, 60.0, 180.0)
    ref = O.run_alg1(M, K, [E], VOXEL, angles_deg=angles)
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, angle_batch=1) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants([E], K)
        ns, kb, kz = ctx.zfirst_plan(0)
        assert 0 < ns < nz and kz == nz // ns == 3
        host = ctx.run(angles)
        dev = torch.empty((1, ny, nx), device="cuda")
        ctx.run(angles, out=dev)
        ctx.check()
        np.testing.assert_array_equal(dev.cpu().numpy(), host)
    iy, ix = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    mask = np.hypot(ix, iy) > 2.5
    a, b = host[0][mask].astype(np.float64), ref[0][mask]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4
    big = mask & (ref[0] > 1e-4 * ref[0][mask].max())
    assert (np.abs(host[0] - ref[0])[big] / ref[0][big]).max() < 2e-3
    np.testing.assert_allclose(host[0][~mask], ref[0][~mask], rtol=1e-4)


SAMPLED = [((64, 512, 512), 4, 0), ((128, 1024, 512), 3, 1), ((32, 512, 2048), 2, 0),
           ((128, 2048, 1024), 2, 0), ((64, 1024, 2048), 2, 1), ((128, 512, 512), 2, 1)]


@pytest.mark.parametrize("shape,c,frame", SAMPLED,
                         ids=["x".join(map(str, s)) + f"c{c}f{f}" for s, c, f in SAMPLED])
def test_sampled_pixels_match_oracle(rsx, shape, c, frame):
    """Every kernel shape of the path: nz = 32, 64, 128 (1, 2 or 4 lanes per
    z line), x rows of 512, 1024, 2048 points, the 512-, 1024- and 2048-row
    selection passes, both frames; 36 angles (two or three passes) averaged
    with the rotation, at sampled output pixels."""
    nz, ny, nx = shape
    E = 280.0
    angles = (0.0, 5.0, 175.0)
    sp = synth.sparse_voxels(shape, c, 3000, seed=43)
    K = synth.optical_constants([E], c, seed=44)
    dev = synth.morphology_sparse_torch(shape, c, sp)
    g = np.random.default_rng(45)
    oy = np.concatenate([[ny // 2, ny // 2 + 1, 3, ny - 2], g.integers(0, ny, 50)])
    ox = np.concatenate([[nx // 2, nx // 2 - 2, 5, nx - 1], g.integers(0, nx, 50)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, frame=frame) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        ns, kb, kz = ctx.zfirst_plan(0)
        assert 0 < ns < nz and kz == min(32, ctx.angle_batch * nz // ns) < 36, (ns, kz)
        out = torch.empty((1, ny, nx), device="cuda")
        ctx.run(angles, out=out)
        ctx.check()
        full = out[0].cpu().numpy().astype(np.float64)
    del dev
    torch.cuda.empty_cache()
    ref = O.run_alg1_sparse_pixels(sp, shape, K[0], E, VOXEL, angles, oy, ox,
                                   uT_mode="literal" if frame == 0 else "lab")
    _sampled_check(full[oy, ox], ref, oy, ox, ny, nx)


def test_energy_beyond_the_plan_takes_the_other_path(rsx):
    """At 175 eV a 32-slice grid reads 25 of its 32 bins: the path steps
    aside for that energy (the multi-angle x pass runs) and serves the next
    one; both energies against the oracle at sampled pixels."""
    shape, c = (32, 512, 1024), 2
    nz, ny, nx = shape
    energies = [175.0, 285.0]
    angles = (0.0, 45.0, 135.0)
    sp = synth.sparse_voxels(shape, c, 2000, seed=46)
    K = synth.optical_constants(energies, c, seed=47)
    dev = synth.morphology_sparse_torch(shape, c, sp)
    g = np.random.default_rng(48)
    oy = np.concatenate([[ny // 2, 2], g.integers(0, ny, 40)])
    ox = np.concatenate([[nx // 2, nx - 3], g.integers(0, nx, 40)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants(energies, K)
        assert ctx.zfirst_plan(0)[0] == 0 and ctx.zfirst_plan(1)[0] > 0
        out = torch.empty((2, ny, nx), device="cuda")
        ctx.run(angles, out=out)
        ctx.check()
        full = out.cpu().numpy().astype(np.float64)
    for ie, E in enumerate(energies):
        ref = O.run_alg1_sparse_pixels(sp, shape, K[ie], E, VOXEL, angles, oy, ox)
        _sampled_check(full[ie][oy, ox], ref, oy, ox, ny, nx)


def test_result_is_bitwise_independent_of_the_angle_batch(rsx):
    """Each angle's planes, transforms and image are the same arithmetic
    whatever pass it falls in: angle_batch 1 (3 angles per pass) and 8
    (18 per pass) give identical images."""
    shape, c = (32, 512, 1024), 3
    nz, ny, nx = shape
    M = synth.morphology_random(shape, c, seed=49, dtype=np.float32)
    energies = [270.0, 300.0]
    K = synth.optical_constants(energies, c, seed=50)
    dev = torch.from_numpy(M).cuda()
    outs = []
    for k in (1, 8):
        with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, angle_batch=k) as ctx:
            ctx.set_morphology(dev)
            ctx.set_optical_constants(energies, K)
            ns = ctx.zfirst_plan(0)[0]
            assert ctx.zfirst_plan(0)[2] == min(32, k * nz // ns)
            out = torch.empty((2, ny, nx), device="cuda")
            ctx.run((0.0, 10.0, 170.0), out=out)
            ctx.check()
            outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
