"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every row of the hot path is checked on its own (polarisation, 3-D FFT,
Ewald projection, detector rotation), then the fused per-angle pipeline and
the whole of Algorithm 1, on seeded inputs at sizes the oracle finishes in
seconds: several FFT tiles, ragged z extents, Nz = 1 films, ny = 1 and a
single voxel.  The full benchmark size (1024 x 1024 x 128, c = 4, FP32) is
checked through a property that holds at any size.

Tolerances (derived in the design notes from the arithmetic):
  FP64: relative L2 error <= 1e-10 over pixels away from q = 0, and
        per-pixel relative <= 1e-8 where X > 1e-8 max X.
  FP32: relative L2 error <= 1e-4 over pixels away from q = 0, and
        per-pixel relative <= 2e-3 where X > 1e-4 max X.
"""
import math

import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O
from paper_2209_13121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {64: dict(norm=1e-10, pix=1e-8, floor=1e-8), 32: dict(norm=1e-4, pix=2e-3, floor=1e-4)}
ENERGIES = [270.0, 285.0, 310.0]
VOXEL = 5.0


@pytest.fixture(scope="module")
def rsx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx as R
    return R


def _real(prec):
    return np.float32 if prec == 32 else np.float64


def _tdtype(prec):
    return torch.float32 if prec == 32 else torch.float64


def _inputs(shape, c, prec, seed):
    M = synth.morphology_random(shape, c, seed=seed, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=seed + 100)
    return M, K


def _center_mask(ny, nx, r=1.5):
    iy, ix = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    return np.hypot(ix, iy) > r


def assert_image_close(gpu, ref, prec, mask=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    t = TOL[prec]
    if mask is None:
        mask = _center_mask(*ref.shape[-2:])
    mask = np.broadcast_to(mask, ref.shape)
    a, b = gpu[mask], ref[mask]
    if b.size and np.abs(b).max() > 0:
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= t["norm"], f"relative L2 error {rel:.3e} > {t['norm']:.0e}"
    big = np.abs(ref) > t["floor"] * np.abs(ref).max()
    if big.any():
        pix = (np.abs(gpu - ref)[big] / np.abs(ref)[big]).max()
        assert pix <= t["pix"], f"per-pixel relative error {pix:.3e} > {t['pix']:.0e}"
    assert np.all(np.isfinite(gpu))


CASES = [
    ((4, 8, 8), 2),
    ((5, 16, 32), 3),     # ragged nz, nx != ny
    ((16, 32, 32), 4),
    ((1, 64, 64), 2),     # 2-D film, Nz = 1
    ((3, 128, 16), 3),    # nx < ny, several y tiles
    ((2, 1, 8), 2),       # ny = 1
    ((1, 1, 1), 1),       # single voxel
    ((7, 4, 2048), 2),    # nx at the x-FFT tile size, ragged nz
    ((6, 32, 128), 3),    # ragged nz
    ((9, 128, 64), 2),    # odd nz
    ((3, 256, 32), 4),    # tall column tile
    ((3, 8, 1024), 3),    # four-step x pass (nx = 1024)
    ((2, 1024, 16), 2),   # four-step y pass (ny = 1024)
    ((4, 6, 8), 2),       # the 8 x 6 x 4 parity grid: ny = 6 (radices 2 and 3)
    ((3, 12, 10), 3),     # nx = 10, ny = 12 (radix 5; 4 x 3)
    ((2, 9, 15), 2),      # odd lateral sizes: 9 = 3 x 3, 15 = 5 x 3 (odd pixel count)
    ((5, 7, 14), 2),      # radix 7, ragged nz
    ((1, 11, 13), 2),     # primes above 7 (the O(p) passes), 2-D film
    ((2, 100, 96), 3),    # 100 = 4 x 5 x 5, 96 = 16 x 2 x 3
]
IDS = ["x".join(map(str, s)) + f"c{c}" for s, c in CASES]


def _ctx(rsx, shape, c, prec, frame=0, **kw):
    nz, ny, nx = shape
    return rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, frame=frame, **kw)


# ------------------------------------------------------------ row a2 + a3
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape,c", CASES, ids=IDS)
def test_polarization_matches_oracle(rsx, shape, c, prec):
    M, K = _inputs(shape, c, prec, seed=1)
    with _ctx(rsx, shape, c, prec) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        p = torch.empty((3,) + shape + (2,), dtype=_tdtype(prec), device="cuda")
        for ie, alpha in ((0, 0.0), (1, 0.9), (2, 2.7)):
            ctx.polarization(ie, alpha, p)
            torch.cuda.synchronize()
            got = p.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            ref = O.rotate_back(O.polarization(M, K[ie], O.e_field(alpha)), alpha)
            # the oracle forms N_rot N_rot - I from entries of size ~1, so its
            # own rounding is ~eps / (4 pi) even where p is small
            scale = max(np.abs(ref).max(), 1.0 / (4 * np.pi))
            tol = 1e-13 if prec == 64 else 3e-7
            np.testing.assert_allclose(got, ref, rtol=0, atol=tol * scale)
            # the optical contrast (ref minus its mean) is also resolved
            d_got, d_ref = got - ref.mean(), ref - ref.mean()
            if np.abs(d_ref).max() > 0:
                rel = np.linalg.norm(d_got - d_ref) / np.linalg.norm(d_ref)
                assert rel < (1e-10 if prec == 64 else 2e-3)


def _wide_angles(M, seed):
    """Euler angles outside [0, 2 pi) x [0, pi] (Sec. 3.1 does not restrict
    them): phi ~ U[-4 pi, 4 pi], theta ~ U[-pi, 2 pi], and one voxel in 16
    with |phi| and |theta| near 100."""
    g = np.random.default_rng(seed)
    M = M.copy()
    shp = M.shape[:-1]
    M[..., 2] = g.uniform(-4 * np.pi, 4 * np.pi, shp)
    M[..., 3] = g.uniform(-np.pi, 2 * np.pi, shp)
    far = g.random(shp) < 1.0 / 16
    M[..., 2][far] = g.choice([-1.0, 1.0], far.sum()) * g.uniform(99.0, 101.0, far.sum())
    M[..., 3][far] = g.choice([-1.0, 1.0], far.sum()) * g.uniform(99.0, 101.0, far.sum())
    return M


WIDE = [((3, 16, 32), 3), ((2, 8, 1024), 4), ((2, 64, 512), 2), ((2, 1024, 64), 2)]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape,c", WIDE, ids=["x".join(map(str, s)) for s, _ in WIDE])
def test_wide_euler_angles_match_oracle(rsx, shape, c, prec):
    """Angles far outside one turn through rsx_polarization and the fused
    per-angle path (for nx = 1024 and 512 in FP32: the bulk-copy x pass),
    at the usual tolerances."""
    M, K = _inputs(shape, c, prec, seed=51)
    M = _wide_angles(M, seed=52)
    with _ctx(rsx, shape, c, prec) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        p = torch.empty((3,) + shape + (2,), dtype=_tdtype(prec), device="cuda")
        img = torch.empty(shape[1:], dtype=_tdtype(prec), device="cuda")
        for ie, alpha in ((0, 0.4), (2, 2.3)):
            ctx.polarization(ie, alpha, p)
            got = p.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            ref = O.rotate_back(O.polarization(M, K[ie], O.e_field(alpha)), alpha)
            scale = max(np.abs(ref).max(), 1.0 / (4 * np.pi))
            np.testing.assert_allclose(got, ref, rtol=0,
                                       atol=(1e-13 if prec == 64 else 3e-7) * scale)
            ctx.scatter_angle(ie, alpha, img)
            ref_img = O.scatter_one_angle(M, K[ie], ENERGIES[ie], VOXEL, alpha)
            assert_image_close(img.cpu().numpy(), ref_img, prec)


@pytest.mark.parametrize("prec", [32, 64])
def test_polarization_lab_frame(rsx, prec):
    shape, c = (3, 8, 16), 3
    M, K = _inputs(shape, c, prec, seed=2)
    with _ctx(rsx, shape, c, prec, frame=rsx.RSX_FRAME_LAB) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        p = torch.empty((3,) + shape + (2,), dtype=_tdtype(prec), device="cuda")
        ctx.polarization(1, 1.1, p)
        got = p.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
        ref = O.polarization(M, K[1], O.e_field(1.1))
        np.testing.assert_allclose(got, ref, rtol=0,
                                   atol=(1e-13 if prec == 64 else 3e-7) * np.abs(ref).max())


# ------------------------------------------------------------------ row a4
FFT_SHAPES = [(2, 2048, 16), (2048, 2, 8), (3, 2048, 4),
              (4, 6, 8), (3, 12, 10), (5, 9, 15), (2, 11, 13), (7, 5, 3), (6, 100, 36),
              (3, 1, 17), (2, 3, 1031), (2, 1031, 2), (1, 4095, 3),
              (4, 8, 8), (5, 16, 32), (1, 64, 64), (3, 128, 16), (2, 1, 8), (1, 1, 1),
              (7, 4, 2048), (16, 32, 32), (6, 2, 4), (3, 4, 1024), (2, 1024, 8)]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape", FFT_SHAPES, ids=["x".join(map(str, s)) for s in FFT_SHAPES])
def test_fft3d_matches_oracle(rsx, shape, prec):
    g = np.random.default_rng(3)
    p = (g.standard_normal((3,) + shape) + 1j * g.standard_normal((3,) + shape))
    dev = torch.from_numpy(np.stack([p.real, p.imag], axis=-1).astype(_real(prec))).cuda()
    with _ctx(rsx, shape, 1, prec) as ctx:
        ctx.fft3d(dev)
        got = dev.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    ref = O.fft3(p.astype(np.complex64 if prec == 32 else np.complex128).astype(np.complex128))
    tol = 1e-12 if prec == 64 else 2e-6
    n = np.prod(shape)
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * math.sqrt(n) * max(1.0, math.log2(n)))


# ------------------------------------------------------------------ row a5
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape", [(4, 8, 8), (5, 16, 32), (1, 64, 64), (3, 128, 16)],
                         ids=["4x8x8", "5x16x32", "1x64x64", "3x128x16"])
def test_ewald_matches_oracle(rsx, shape, prec):
    M, K = _inputs(shape, 2, 64, seed=4)
    pt = O.fft3(O.polarization(M, K[0], O.e_field(0.3)))
    dev = torch.from_numpy(np.stack([pt.real, pt.imag], axis=-1).astype(_real(prec))).cuda()
    with _ctx(rsx, shape, 2, prec) as ctx:
        ctx.set_optical_constants(ENERGIES, K)
        for ie in range(3):
            img = torch.empty(shape[1:], dtype=_tdtype(prec), device="cuda")
            ctx.ewald(ie, dev, img)
            ref = O.fftshift2(O.ewald(pt, ENERGIES[ie], VOXEL))
            assert_image_close(img.cpu().numpy(), ref, prec)


def test_ewald_outside_sphere_is_zero(rsx):
    shape = (2, 16, 16)
    pt = np.ones((3,) + shape, complex)
    dev = torch.from_numpy(np.stack([pt.real, pt.imag], axis=-1)).cuda()
    with rsx.Context(16, 16, 2, 1, 2.0, precision=64) as ctx:
        ctx.set_optical_constants([120.0], np.zeros((1, 1, 4)))
        img = torch.empty((16, 16), dtype=torch.float64, device="cuda")
        ctx.ewald(0, dev, img)
        ref = O.fftshift2(O.ewald(pt, 120.0, 2.0))
        got = img.cpu().numpy()
        assert np.array_equal(got == 0, ref == 0) and (ref == 0).sum() > 20
        np.testing.assert_allclose(got, ref, rtol=1e-12)


# ------------------------------------------------------------------ row a6
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("ny,nx", [(16, 16), (32, 8), (1, 8), (64, 128)])
def test_rotate_accumulate_matches_oracle(rsx, ny, nx, prec):
    g = np.random.default_rng(5)
    img = g.random((ny, nx))
    acc0 = g.random((ny, nx))
    with rsx.Context(nx, ny, 1, 1, VOXEL, precision=prec) as ctx:
        for alpha in (0.0, 0.35, math.pi / 2, 2.9):
            d_img = torch.from_numpy(img.astype(_real(prec))).cuda()
            d_acc = torch.from_numpy(acc0.astype(_real(prec))).cuda()
            ctx.rotate_accumulate(d_img, alpha, d_acc)
            ref = acc0.astype(_real(prec)).astype(np.float64) + O.rotate_image(
                img.astype(_real(prec)).astype(np.float64), alpha)
            tol = 1e-12 if prec == 64 else 2e-6
            np.testing.assert_allclose(d_acc.cpu().numpy(), ref, rtol=tol, atol=tol)


# ----------------------------------------------- rows a1-a5 fused (hot path)
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape,c", CASES, ids=IDS)
def test_scatter_angle_matches_oracle(rsx, shape, c, prec):
    M, K = _inputs(shape, c, prec, seed=6)
    with _ctx(rsx, shape, c, prec) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        img = torch.empty(shape[1:], dtype=_tdtype(prec), device="cuda")
        for ie, alpha in ((0, 0.0), (1, 0.7), (2, 3.0)):
            ctx.scatter_angle(ie, alpha, img)
            ref = O.scatter_one_angle(M, K[ie], ENERGIES[ie], VOXEL, alpha)
            assert_image_close(img.cpu().numpy(), ref, prec)
            # q = 0 itself (the constant part returns there)
            ny, nx = shape[1:]
            np.testing.assert_allclose(img.cpu().numpy()[ny // 2, nx // 2], ref[ny // 2, nx // 2],
                                       rtol=1e-10 if prec == 64 else 1e-5)


# Sizes at which the persistent FP32 passes give each block several work
# items: x rows (nx = 1024: groups of two rows and an odd tail) and y tiles
# (ny = 1024: both input buffers refilled more than once); the fused y+z
# pass at its edges: nz = 1 (both q_z bins are plane 0), the narrowest
# width (one tile pair), a field split between two block pairs, a 2048-wide
# grid (Stockham x pass feeding the fused y+z pass); one component (one
# bulk-copy stage per row); 512-row grids (the 16-column variant of the
# fused pass, with items split between blocks); 512-wide rows (the 32 x 16
# transform of the bulk-copy x pass) with one and three components, alone
# and feeding the 512-row fused pass.
MULTI = [((2, 2048, 16), 2), ((1, 2048, 64), 3), ((4, 2048, 32), 2), ((8, 2048, 128), 2),
         ((3, 256, 1024), 2), ((8, 1024, 256), 2), ((1, 1024, 64), 3), ((4, 1024, 16), 2),
         ((2, 1024, 512), 2), ((1, 1024, 2048), 2), ((3, 8, 1024), 1), ((4, 512, 64), 2),
         ((2, 512, 1024), 2), ((5, 64, 512), 3), ((3, 8, 512), 1), ((4, 512, 512), 2)]


@pytest.mark.parametrize("shape,c", MULTI, ids=["x".join(map(str, s)) for s, _ in MULTI])
def test_scatter_angle_persistent_passes(rsx, shape, c):
    M, K = _inputs(shape, c, 32, seed=16)
    with _ctx(rsx, shape, c, 32) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        img = torch.empty(shape[1:], dtype=torch.float32, device="cuda")
        for ie, alpha in ((0, 0.3), (2, 2.0)):
            ctx.scatter_angle(ie, alpha, img)
            ref = O.scatter_one_angle(M, K[ie], ENERGIES[ie], VOXEL, alpha)
            assert_image_close(img.cpu().numpy(), ref, 32)


@pytest.mark.parametrize("ny", [1024, 2048])
@pytest.mark.parametrize("frame", [0, 1])
def test_fused_yz_pass_off_sphere_pixels_and_frames(rsx, frame, ny):
    """ny = 1024 and 2048 with 2 nm voxels at 270 eV: the detector corners
    lie outside the Ewald sphere (zero in both paths), in either frame."""
    shape, c, vox = (4, ny, 32), 2, 2.0
    M, K = _inputs(shape, c, 32, seed=18)
    nz, ny, nx = shape
    with rsx.Context(nx, ny, nz, c, vox, precision=32, frame=frame) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        img = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        ctx.scatter_angle(0, 0.6, img)
        got = img.cpu().numpy()
    ref = O.scatter_one_angle(M, K[0], ENERGIES[0], vox, 0.6,
                              uT_mode="literal" if frame == 0 else "lab")
    assert (ref == 0).sum() > 100
    assert np.array_equal(got == 0, ref == 0)
    assert_image_close(got, ref, 32)


# ------------------------------------------------------- Algorithm 1 (a7)
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape,c", CASES[:5], ids=IDS[:5])
def test_run_matches_oracle(rsx, shape, c, prec):
    M, K = _inputs(shape, c, prec, seed=7)
    angles = (0.0, 30.0, 180.0)
    ref = O.run_alg1(M, K, ENERGIES, VOXEL, angles_deg=angles)
    with _ctx(rsx, shape, c, prec) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        host = ctx.run(angles)
        dev = torch.empty(ref.shape, dtype=_tdtype(prec), device="cuda")
        ctx.run(angles, out=dev)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dev.cpu().numpy(), host)
    mask = _center_mask(*shape[1:], r=2.5)
    assert_image_close(host, ref, prec, mask=mask)
    center = ~mask
    np.testing.assert_allclose(host[:, center], ref[:, center], rtol=1e-9 if prec == 64 else 1e-4)


ODD = [((4, 6, 8), 2), ((3, 12, 10), 3), ((2, 9, 15), 2), ((3, 25, 48), 2), ((1, 45, 35), 2),
       ((2, 16, 12), 2), ((2, 3, 4093), 1), ((2, 4, 4096), 2)]   # the largest rows: prime, 2^12


@pytest.mark.parametrize("algorithm", [1, 2, 3])
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("shape,c", ODD, ids=["x".join(map(str, s)) for s, _ in ODD])
def test_run_non_power_of_two_grids(rsx, shape, c, prec, algorithm):
    """Any nx and ny (Sec. 3.3 step 4 puts no restriction on the grid): the
    P0 parity grid 8 x 6 x 4 and other lateral sizes with factors 3, 5 and
    7, through rsx_run for Algorithm 1, Algorithm 2 and the linearity path,
    host and device output, against the oracle."""
    M, K = _inputs(shape, c, prec, seed=71)
    angles = (0.0, 45.0, 180.0)
    nz, ny, nx = shape
    ref = O.run_alg1(M, K, ENERGIES, VOXEL, angles_deg=angles)
    with _ctx(rsx, shape, c, prec, algorithm=algorithm) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        host = ctx.run(angles)
        dev = torch.empty(ref.shape, dtype=_tdtype(prec), device="cuda")
        ctx.run(angles, out=dev)
        ctx.check()
        np.testing.assert_array_equal(dev.cpu().numpy(), host)
    assert_image_close(host, ref, prec, mask=_center_mask(ny, nx, r=2.5))


BATCHED = [((2, 512, 512), 3, 4), ((1, 1024, 1024), 2, 3), ((2, 512, 1024), 2, 8),
           ((2, 1024, 512), 2, 2), ((3, 64, 1024), 3, 4), ((2, 32, 2048), 2, 2),
           ((3, 16, 2048), 4, 1), ((2, 8, 2048), 3, 3), ((3, 1024, 512), 2, 4),
           ((2, 2048, 512), 2, 4)]


@pytest.mark.parametrize("frame", [0, 1])
@pytest.mark.parametrize("shape,c,kx", BATCHED, ids=["x".join(map(str, s)) + f"k{k}"
                                                    for s, _, k in BATCHED])
def test_run_batched_angles_match_oracle(rsx, shape, c, kx, frame):
    """Algorithm 1 with the morphology read once per batch of angles (the
    multi-angle x pass, FP32): seven angles, so the last batch is partial,
    against the oracle; and against the same context shape with one angle
    per pass."""
    M, K = _inputs(shape, c, 32, seed=61)
    angles = (0.0, 30.0, 180.0)
    nz, ny, nx = shape
    ref = O.run_alg1(M, K[:1], ENERGIES[:1], VOXEL, angles_deg=angles,
                     uT_mode="literal" if frame == 0 else "lab")
    dev = torch.from_numpy(M).cuda()
    outs = {}
    for k in (kx, 1):
        with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, frame=frame, angle_batch=k) as ctx:
            assert ctx.angle_batch == k
            ctx.set_morphology(dev)
            ctx.set_optical_constants(ENERGIES[:1], K[:1])
            out = torch.empty((1, ny, nx), device="cuda")
            ctx.run(angles, out=out)
            ctx.check()
            outs[k] = out.cpu().numpy()
    mask = _center_mask(ny, nx, r=2.5)
    assert_image_close(outs[kx], ref, 32, mask=mask)
    assert_image_close(outs[kx], outs[1], 32, mask=mask)


def test_angle_batch_applies_only_where_the_multi_angle_pass_runs(rsx):
    for shape, prec, alg, want in (((4, 1024, 1024), 32, 1, 8), ((4, 1024, 1024), 64, 1, 1),
                                   ((1024, 1024, 1024), 32, 1, 1), ((512, 1024, 1024), 32, 1, 2),
                                   ((4, 1024, 1024), 32, 2, 1), ((3, 1024, 1024), 32, 1, 8),
                                   ((4, 256, 1024), 32, 1, 8), ((4, 64, 2048), 32, 1, 3),
                                   ((2, 64, 1000), 32, 1, 1), ((4, 64, 2048), 64, 1, 1)):
        nz, ny, nx = shape
        cfg = rsx.make_config(nx, ny, nz, 2, VOXEL, precision=prec, algorithm=alg)
        # the batch of a context, without allocating the large ones
        if nz >= 512:
            one = rsx.workspace_bytes(rsx.make_config(nx, ny, nz, 2, VOXEL, angle_batch=1))
            assert rsx.workspace_bytes(cfg) == one + (want - 1) * 3 * nx * ny * nz * 8
            continue
        with rsx.Context(nx, ny, nz, 2, VOXEL, precision=prec, algorithm=alg) as ctx:
            assert ctx.angle_batch == want, (shape, prec, alg)


@pytest.mark.parametrize("prec", [32, 64])
def test_run_lab_frame_and_rotation_off(rsx, prec):
    shape, c = (4, 16, 16), 3
    M, K = _inputs(shape, c, prec, seed=8)
    with _ctx(rsx, shape, c, prec, frame=rsx.RSX_FRAME_LAB) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        got = ctx.run((0.0, 45.0, 135.0))
        ref = O.run_alg1(M, K, ENERGIES, VOXEL, angles_deg=(0.0, 45.0, 135.0), uT_mode="lab")
        assert_image_close(got, ref, prec, mask=_center_mask(16, 16, 2.5))
        off = ctx.run((0.0, 45.0, 135.0), rotation=False)
        ref_off = O.run_alg1(M, K, ENERGIES, VOXEL, rotation=False, uT_mode="lab")
        assert_image_close(off, ref_off, prec)


def test_energy_shards_are_bitwise_rows_of_full_run(rsx):
    """Sharding energies across ranks (independent units, no collective)
    gives exactly the rows of the unsharded run."""
    shape, c = (4, 32, 32), 4
    E = list(np.linspace(270, 310, 6))
    M = synth.morphology_random(shape, c, seed=9)
    K = synth.optical_constants(E, c, seed=10)
    with _ctx(rsx, shape, c, 32) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(E, K)
        full = ctx.run((0, 20, 180))
        parts = [ctx.run((0, 20, 180), energy_indices=idx) for idx in ([0, 1, 2], [3, 4], [5])]
    np.testing.assert_array_equal(np.concatenate(parts), full)


def test_device_morphology_is_borrowed(rsx):
    shape, c = (3, 16, 32), 2
    M, K = _inputs(shape, c, 32, seed=11)
    with _ctx(rsx, shape, c, 32) as a, _ctx(rsx, shape, c, 32) as b:
        a.set_morphology(M)
        b.set_morphology(torch.from_numpy(M).cuda())
        for x in (a, b):
            x.set_optical_constants(ENERGIES, K)
        np.testing.assert_array_equal(a.run((0, 60, 120)), b.run((0, 60, 120)))


def test_async_upload_pipeline_matches_synchronous_upload(rsx):
    """Two contexts on two streams, the next morphology uploaded
    asynchronously from page-locked memory while the other context runs:
    every energy's image equals the synchronous single-context result."""
    shape, c = (4, 32, 64), 3
    Ms = [_inputs(shape, c, 32, seed=40 + i)[0] for i in range(3)]
    _, K = _inputs(shape, c, 32, seed=40)
    pinned = []
    for M in Ms:
        t = torch.empty(M.shape, dtype=torch.float32, pin_memory=True)
        t.copy_(torch.from_numpy(M))
        pinned.append(t)
    ref = []
    with _ctx(rsx, shape, c, 32) as a:
        a.set_optical_constants(ENERGIES, K)
        for i, M in enumerate(Ms):
            a.set_morphology(M)
            ref.append(a.run((0, 30, 180), energy_indices=[i]))
    got = []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    with _ctx(rsx, shape, c, 32) as a, _ctx(rsx, shape, c, 32) as b:
        cx = [a, b]
        for x in cx:
            x.set_optical_constants(ENERGIES, K)
        cx[0].set_morphology(pinned[0].numpy(), stream=streams[0], async_copy=True)
        for i in range(3):
            if i + 1 < 3:
                j = (i + 1) % 2
                cx[j].set_morphology(pinned[i + 1].numpy(), stream=streams[j], async_copy=True)
            got.append(cx[i % 2].run((0, 30, 180), energy_indices=[i], stream=streams[i % 2]))
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


def test_async_upload_needs_page_locked_memory(rsx):
    shape, c = (2, 8, 8), 2
    M, K = _inputs(shape, c, 32, seed=41)
    with _ctx(rsx, shape, c, 32) as a:
        with pytest.raises(rsx.RsxError) as e:
            a.set_morphology(M, async_copy=True)   # pageable numpy memory
        assert e.value.code == rsx.RSX_ERR_INVALID


# ------------------------------------------------------------- error paths
@pytest.mark.parametrize("algorithm", [1, 2, 3])
def test_pipeline_wait_timeout_is_reported_and_recoverable(rsx, algorithm):
    """The pipelined kernels' copy waits are bounded.  With a bound of zero
    polls every such wait runs out at once: each kernel gives up cleanly (its
    copies in flight drained under the default bound), the run reports
    RSX_ERR_CUDA without touching its host output, and with the default
    bound restored the same context gives the same result as a fresh one.
    No fault is involved."""
    shape, c = (2, 1024, 1024), 2   # FP32, nx = ny = 1024: bulk-copy x pass, fused y+z pass
    nz, ny, nx = shape
    M, K = _inputs(shape, c, 32, seed=22)
    dev = torch.from_numpy(M).cuda()
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, algorithm=algorithm) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants(ENERGIES[:1], K[:1])
        ref = ctx.run((0.0, 90.0, 90.0))
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, algorithm=algorithm) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants(ENERGIES[:1], K[:1])
        ctx.set_wait_limit(0)   # before the energy's first run: per-energy passes run too
        out = np.full((1, ny, nx), 7.0, dtype=np.float32)
        with pytest.raises(rsx.RsxError) as e:
            ctx.run((0.0, 90.0, 90.0), out=out)
        assert e.value.code == rsx.RSX_ERR_CUDA and "timed out" in str(e.value)
        assert np.all(out == 7.0)   # the failing call left its host output untouched
        ctx.set_wait_limit()
        np.testing.assert_array_equal(ctx.run((0.0, 90.0, 90.0)), ref)
        # device output: the call returns before the GPU is done, so the
        # timeout is reported by rsx_check, which also drops the per-energy
        # data an aborted kernel produced
        dout = torch.full((1, ny, nx), 7.0, device="cuda")
        ctx.set_optical_constants(ENERGIES[:1], K[:1])   # drops the per-energy data
        ctx.set_wait_limit(0)
        ctx.run((0.0, 90.0, 90.0), out=dout)
        with pytest.raises(rsx.RsxError) as e:
            ctx.check()
        assert e.value.code == rsx.RSX_ERR_CUDA and "timed out" in str(e.value)
        ctx.check()   # the flag was cleared by the report
        ctx.set_wait_limit()
        ctx.run((0.0, 90.0, 90.0), out=dout)
        ctx.check()
        np.testing.assert_array_equal(dout.cpu().numpy(), ref)



def test_errors_are_reported_and_write_nothing(rsx):
    shape, c = (2, 8, 8), 2
    M, K = _inputs(shape, c, 32, seed=12)
    with _ctx(rsx, shape, c, 32, validate=True) as ctx:
        out = np.full((1, 8, 8), 7.0, dtype=np.float32)
        with pytest.raises(rsx.RsxError) as e:   # no morphology yet
            ctx.run((0, 10, 20), out=out, energy_indices=[0])
        assert e.value.code == rsx.RSX_ERR_STATE
        assert np.all(out == 7.0)
        bad = M.copy()
        bad[1, 0, 0, 0, 1] = 1.5  # s > 1 (Sec. 3.1)
        with pytest.raises(rsx.RsxError) as e:
            ctx.set_morphology(bad)
        assert e.value.code == rsx.RSX_ERR_INVALID
        with pytest.raises(rsx.RsxError) as e:
            ctx.set_morphology(torch.from_numpy(bad).cuda())
        assert e.value.code == rsx.RSX_ERR_INVALID
        nanm = M.copy()
        nanm[0, 1, 2, 3, 2] = np.nan
        with pytest.raises(rsx.RsxError):
            ctx.set_morphology(nanm)
        ctx.set_morphology(M)
        with pytest.raises(rsx.RsxError) as e:
            ctx.set_optical_constants([285.0, -1.0, 300.0], K)
        assert e.value.code == rsx.RSX_ERR_INVALID
        ctx.set_optical_constants(ENERGIES, K)
        for kw in (dict(angles=(0, 0, 10)), dict(angles=(10, 1, 0)),
                   dict(energy_indices=[3]), dict(energy_indices=[-1])):
            o = np.full((len(kw.get("energy_indices", ENERGIES)), 8, 8), 7.0, dtype=np.float32)
            with pytest.raises(rsx.RsxError) as e:
                ctx.run(kw.get("angles", (0, 10, 20)), energy_indices=kw.get("energy_indices"),
                        out=o)
            assert e.value.code == rsx.RSX_ERR_INVALID
            assert np.all(o == 7.0)
        empty = ctx.run((0, 10, 20), energy_indices=[])
        assert empty.shape == (0, 8, 8)


def test_device_entry_points_refuse_host_pointers(rsx):
    """A host address where device memory is expected is refused by the C
    entry points (cudaPointerGetAttributes) before anything is enqueued."""
    shape, c = (2, 8, 8), 2
    M, K = _inputs(shape, c, 32, seed=14)
    host_p = np.zeros((3,) + shape + (2,), np.float32)
    host_img = np.zeros(shape[1:], np.float32)
    dev_img = torch.zeros(shape[1:], device="cuda")
    with _ctx(rsx, shape, c, 32) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        calls = [lambda: ctx.polarization(0, 0.0, host_p.ctypes.data),
                 lambda: ctx.fft3d(host_p.ctypes.data),
                 lambda: ctx.scatter_angle(0, 0.0, host_img.ctypes.data),
                 lambda: ctx.rotate_accumulate(host_img.ctypes.data, 0.0, dev_img),
                 lambda: ctx.ewald(0, host_p.ctypes.data, dev_img),
                 lambda: ctx.set_morphology(host_p.ctypes.data)]
        for call in calls:
            with pytest.raises((rsx.RsxError, ValueError)) as e:
                call()
            if isinstance(e.value, rsx.RsxError):
                assert e.value.code == rsx.RSX_ERR_INVALID
        lib = rsx.lib()
        import ctypes
        rc = lib.rsx_run(ctx._h, 0.0, 10.0, 20.0, 1, None, 3, ctypes.c_void_p(host_img.ctypes.data),
                         rsx.RSX_DEVICE, None)
        assert rc == rsx.RSX_ERR_INVALID
        assert "host memory" in lib.rsx_last_error().decode()
        # the context still works
        ctx.scatter_angle(0, 0.0, dev_img)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(dev_img.cpu().numpy()))


@pytest.mark.parametrize("algorithm", [1, 3])
def test_fp64_tall_stack_pruned_z_transform(rsx, algorithm):
    """FP64 with nz = 4096 (the z twiddle table then needs 64 KB of shared
    memory) on a lateral grid the bulk-copy Ewald kernel does not take:
    the pruned z transform (Algorithm 1) and the linearity path's q_z bins
    (Algorithm 3) against the oracle."""
    shape, c = (4096, 4, 8), 2
    M, K = _inputs(shape, c, 64, seed=15)
    angles = (0.0, 90.0, 90.0)
    ref = O.run_alg1(M, K, ENERGIES[:1], VOXEL, angles_deg=angles)
    nz, ny, nx = shape
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=64, algorithm=algorithm) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES[:1], K[:1])
        got = ctx.run(angles)
    assert_image_close(got, ref, 64, mask=_center_mask(ny, nx, 0.5))


def test_unvalidated_context_accepts_out_of_range_v_sum(rsx):
    """Sec. 3.1: the sum of v over components is never checked."""
    shape, c = (1, 8, 8), 2
    M, K = _inputs(shape, c, 64, seed=13)
    M[..., 0] = 1.0  # every component fills every voxel: sum 2
    with _ctx(rsx, shape, c, 64, validate=True) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        got = ctx.run((0, 90, 90))
    ref = O.run_alg1(M, K, ENERGIES, VOXEL, angles_deg=(0, 90, 90))
    assert_image_close(got, ref, 64, mask=_center_mask(8, 8, 2.5))


# ------------------------------- full benchmark size (sampled pixels, exact)
@pytest.mark.parametrize("algorithm", [1, 2])
def test_full_size_sampled_pixels_match_oracle(rsx, algorithm):
    """At the benchmark's size and launch configuration (1024 x 1024 x 128,
    c = 4, FP32: the bulk-copy x pass and the fused y+z pass), a morphology
    that is vacuum except at ~20000 random voxels: detector pixels of two
    angles, sampled, against the oracle's sampled path (exact by linearity
    of the DFT, pinned against the full path)."""
    if torch.cuda.get_device_properties(0).total_memory < 40e9:
        pytest.skip("needs ~20 GB of device memory")
    shape, c, E = (128, 1024, 1024), 4, 285.0
    nz, ny, nx = shape
    sp = synth.sparse_voxels(shape, c, 20000, seed=19)
    K = synth.optical_constants([E], c, seed=20)
    dev = synth.morphology_sparse_torch(shape, c, sp)
    g = np.random.default_rng(21)
    iy = np.concatenate([[0, 0, 1, 5, ny - 1, 300], g.integers(0, ny, 120)])
    ix = np.concatenate([[0, 1, 0, 7, 3, nx - 2], g.integers(0, nx, 120)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, algorithm=algorithm) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        img = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        for alpha in (0.0, 1.1):
            ctx.scatter_angle(0, alpha, img)
            full = img.cpu().numpy().astype(np.float64)
            got = full[(iy + ny // 2) % ny, (ix + nx // 2) % nx]
            ref = O.scatter_sparse_pixels(sp, shape, K[0], E, VOXEL, alpha, iy, ix)
            center = (iy == 0) & (ix == 0)
            np.testing.assert_allclose(got[center], ref[center], rtol=1e-5)
            rest = ~center
            scale = ref[rest].max()
            rel = np.linalg.norm(got[rest] - ref[rest]) / np.linalg.norm(ref[rest])
            assert rel < 1e-4, rel
            big = rest & (ref > 1e-4 * scale)
            assert big.sum() > 100
            assert (np.abs(got - ref)[big] / ref[big]).max() < 2e-3
    del dev
    torch.cuda.empty_cache()


def test_full_size_run_sampled_pixels_match_oracle(rsx):
    """rsx_run at the benchmark's size and launch configuration (1024 x
    1024 x 128, c = 4, FP32, device output: the z-first path with its
    default batch (polarisation + z-FFT, x-FFT of the kept planes, the
    y-FFT selecting each pixel's bins), the Ewald image, the rotation into
    the average), ten angles (one pass of the z-first kernels), against the
    oracle's average at sampled output pixels (each angle's unrotated image
    at the corners the rotation reads, exact by linearity of the DFT)."""
    if torch.cuda.get_device_properties(0).total_memory < 100e9:
        pytest.skip("needs ~45 GB of device memory")
    shape, c, E = (128, 1024, 1024), 4, 285.0
    nz, ny, nx = shape
    angles = (0.0, 2.0, 18.0)
    sp = synth.sparse_voxels(shape, c, 6000, seed=26)
    K = synth.optical_constants([E], c, seed=27)
    dev = synth.morphology_sparse_torch(shape, c, sp)
    g = np.random.default_rng(28)
    oy = np.concatenate([[ny // 2, ny // 2 + 1, 3, ny - 2], g.integers(0, ny, 50)])
    ox = np.concatenate([[nx // 2, nx // 2 - 2, 5, nx - 1], g.integers(0, nx, 50)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32) as ctx:
        assert ctx.angle_batch == 8
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        out = torch.empty((1, ny, nx), dtype=torch.float32, device="cuda")
        ctx.run(angles, out=out)
        ctx.check()
        full = out[0].cpu().numpy().astype(np.float64)
    del dev
    torch.cuda.empty_cache()
    got = full[oy, ox]
    ref = O.run_alg1_sparse_pixels(sp, shape, K[0], E, VOXEL, angles, oy, ox)
    # pixels whose rotated samples reach q = 0 carry its large value
    center = np.hypot(oy - ny // 2, ox - nx // 2) < 2.5
    assert center[:2].all()
    np.testing.assert_allclose(got[center], ref[center], rtol=1e-5)
    rest = ~center
    rel = np.linalg.norm(got[rest] - ref[rest]) / np.linalg.norm(ref[rest])
    assert rel < 1e-4, rel
    big = rest & (ref > 1e-4 * ref[rest].max())
    assert big.sum() > 30
    assert (np.abs(got - ref)[big] / ref[big]).max() < 2e-3


@pytest.mark.parametrize("shape,c,prec", [((1, 2048, 2048), 2, 32), ((1, 2048, 2048), 2, 64),
                                          ((64, 2048, 2048), 4, 32)],
                         ids=["2048x2048x1-f32", "2048x2048x1-f64", "2048x2048x64-f32"])
def test_run_2048_grids_sampled_pixels_match_oracle(rsx, shape, c, prec):
    """rsx_run on the 2048-wide grids of Sec. 5.1 (the 2-D film) and Sec. 6.2
    (2048 x 2048 x 64, c = 4): FP32 through the 2048-point multi-angle x
    pass (the film) or the z-first path (64 slices), FP64 through the
    general kernels; five angles, sampled output pixels against the
    oracle's average (exact by linearity of the DFT)."""
    nz, ny, nx = shape
    E = 280.0
    angles = (0.0, 40.0, 160.0)
    sp = synth.sparse_voxels(shape, c, 4000, seed=29)
    K = synth.optical_constants([E], c, seed=30)
    dev = synth.morphology_sparse_torch(shape, c, sp, dtype=_tdtype(prec))
    g = np.random.default_rng(31)
    oy = np.concatenate([[ny // 2, 7, ny - 3], g.integers(0, ny, 40)])
    ox = np.concatenate([[nx // 2, nx - 1, 11], g.integers(0, nx, 40)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec) as ctx:
        # FP32: 3 angles per multi-angle pass (the film); p buffers within
        # 32 GiB for the z-first path (5 of 6.4 GB at 64 slices)
        assert ctx.angle_batch == (1 if prec == 64 else 3 if nz == 1 else 5)
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        out = torch.empty((1, ny, nx), dtype=_tdtype(prec), device="cuda")
        ctx.run(angles, out=out)
        ctx.check()
        full = out[0].cpu().numpy().astype(np.float64)
    del dev
    torch.cuda.empty_cache()
    got = full[oy, ox]
    ref = O.run_alg1_sparse_pixels(sp, shape, K[0], E, VOXEL, angles, oy, ox)
    center = np.hypot(oy - ny // 2, ox - nx // 2) < 2.5
    t = TOL[prec]
    np.testing.assert_allclose(got[center], ref[center], rtol=1e-5 if prec == 32 else 1e-10)
    rest = ~center
    rel = np.linalg.norm(got[rest] - ref[rest]) / np.linalg.norm(ref[rest])
    assert rel < t["norm"], rel
    big = rest & (ref > t["floor"] * ref[rest].max())
    assert big.sum() > 20
    assert (np.abs(got - ref)[big] / ref[big]).max() < t["pix"]


@pytest.mark.parametrize("shape,c", [((1024, 1024, 16), 2), ((64, 512, 512), 4)])
def test_sampled_pixels_at_the_fused_pass_limits(rsx, shape, c):
    """nz = 1024, the largest the fused y+z pass takes (the whole 227 KB of
    shared memory), and the 512 x 512 x 64, c = 4 grid (the 512-point x
    pass and the 512-row fused pass at their launch shape), vacuum except at
    sparse voxels: sampled pixels against the oracle's sampled path."""
    nz, ny, nx = shape
    E = 285.0
    sp = synth.sparse_voxels(shape, c, 3000, seed=23)
    K = synth.optical_constants([E], c, seed=24)
    dev = synth.morphology_sparse_torch(shape, c, sp)
    g = np.random.default_rng(25)
    iy = np.concatenate([[0, 1, ny - 1], g.integers(0, ny, 60)])
    ix = np.concatenate([[0, 3, nx - 1], g.integers(0, nx, 60)])
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        img = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        ctx.scatter_angle(0, 0.4, img)
        full = img.cpu().numpy().astype(np.float64)
    got = full[(iy + ny // 2) % ny, (ix + nx // 2) % nx]
    ref = O.scatter_sparse_pixels(sp, shape, K[0], E, VOXEL, 0.4, iy, ix)
    rest = ~((iy == 0) & (ix == 0))
    rel = np.linalg.norm(got[rest] - ref[rest]) / np.linalg.norm(ref[rest])
    assert rel < 1e-4, rel
    np.testing.assert_allclose(got[~rest], ref[~rest], rtol=1e-5)


# ------------------------------------------ full benchmark size (property)
def test_full_size_z_uniform_reduces_to_film(rsx):
    """At 1024 x 1024 x 128, c = 4, FP32 (the benchmark's launch shape), a
    morphology uniform along z must give tent(q_z) * Nz^2 * X_film, where
    X_film is the oracle's Nz = 1 image and tent = max(0, 1 - |q_z|/dq_z)
    (linear interpolation between the bracketing q_z bins, Eq. Ewald)."""
    if torch.cuda.get_device_properties(0).total_memory < 40e9:
        pytest.skip("needs ~15 GB of device memory")
    nx = ny = 1024
    nz, c, E = 128, 4, 285.0
    M2 = synth.morphology_random((1, ny, nx), c, seed=14, dtype=np.float32)
    K = synth.optical_constants([E], c, seed=15)
    dev = torch.from_numpy(M2).cuda().expand(c, nz, ny, nx, 4).contiguous()
    k = O.wavenumber(E)
    qx = np.fft.fftshift(O.q_axis(nx, VOXEL))[None, :]
    qy = np.fft.fftshift(O.q_axis(ny, VOXEL))[:, None]
    qz = -k + np.sqrt(k * k - qx * qx - qy * qy)
    tent = np.maximum(0.0, 1.0 - np.abs(qz) / (2 * np.pi / (nz * VOXEL)))
    assert (tent > 0).sum() > 1000
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32) as ctx:
        ctx.set_morphology(dev)
        ctx.set_optical_constants([E], K)
        img = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
        for alpha in (0.0, 0.5):
            ctx.scatter_angle(0, alpha, img)
            film = O.scatter_one_angle(M2, K[0], E, VOXEL, alpha)
            ref = tent * nz ** 2 * film
            assert_image_close(img.cpu().numpy(), ref, 32, mask=_center_mask(ny, nx) & (tent > 0.05))
