"""Algorithms 2 and 3 (memory minimisation, Sec. 4.3) and the linearity
restatement of Algorithm 2, against the CPU oracle.

N_t from Algorithm 3 (device-resident morphology in one pass, or a host
morphology streamed one component at a time in chunks), p = N_t . e, and
whole runs, which must also agree with Algorithm 1."""
import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O
from paper_2209_13121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENERGIES = [272.0, 286.0, 305.0]
VOXEL = 5.0
NT_TOL = {64: 1e-13, 32: 3e-7}   # relative to max(|N_t|, 1/(4 pi)), as for p
TOL = {64: dict(norm=1e-10, pix=1e-8, floor=1e-8), 32: dict(norm=1e-4, pix=2e-3, floor=1e-4)}


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


def _tdt(prec):
    return torch.float32 if prec == 32 else torch.float64


def _close_img(got, ref, prec, r=2.5):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    ny, nx = ref.shape[-2:]
    iy, ix = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    far = np.broadcast_to(np.hypot(ix, iy) > r, ref.shape)
    t = TOL[prec]
    rel = np.linalg.norm((got - ref)[far]) / np.linalg.norm(ref[far])
    assert rel <= t["norm"], rel
    big = ref > t["floor"] * ref.max()
    assert (np.abs(got - ref)[big] / ref[big]).max() <= t["pix"]


def _nt_entries(Nt):
    """Oracle N_t [..., 3, 3] -> the five stored entries [5][...]."""
    return np.stack([Nt[..., 0, 0], Nt[..., 0, 1], Nt[..., 1, 1], Nt[..., 0, 2], Nt[..., 1, 2]])


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("shape,c", [((4, 8, 16), 3), ((5, 32, 32), 4), ((1, 64, 64), 2),
                                     ((2, 1, 8), 1)])
def test_nt_matches_oracle(rsx, shape, c, prec, where):
    M = synth.morphology_random(shape, c, seed=51, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=52)
    nz, ny, nx = shape
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=2) as ctx:
        ctx.set_morphology(M if where == "host" else torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        out = torch.empty((5,) + shape + (2,), dtype=_tdt(prec), device="cuda")
        for ie in (2, 0):
            ctx.nt(ie, out)
            got = out.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            ref = _nt_entries(O.nr_computation(M, K[ie]))
            scale = max(np.abs(ref).max(), 1 / (4 * np.pi))
            np.testing.assert_allclose(got, ref, rtol=0, atol=NT_TOL[prec] * scale)


def test_nt_streamed_in_several_chunks(rsx):
    """A host morphology larger than one staging chunk (2^22 voxels): the
    streamed N_t equals the one-pass device result, checked against the
    oracle on a sample of voxels."""
    shape, c = (80, 256, 256), 2          # 5.2 M voxels: two chunks per component
    nz, ny, nx = shape
    M = synth.morphology_random(shape, c, seed=53)
    K = synth.optical_constants([285.0], c, seed=54)
    outs = []
    for src in (M, torch.from_numpy(M).cuda()):
        with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, algorithm=2) as ctx:
            ctx.set_morphology(src)
            ctx.set_optical_constants([285.0], K)
            out = torch.empty((5,) + shape + (2,), dtype=torch.float32, device="cuda")
            ctx.nt(0, out)
            outs.append(out.cpu().numpy())
    np.testing.assert_allclose(outs[0], outs[1], rtol=0, atol=1e-7)
    g = np.random.default_rng(0)
    flat = g.choice(np.prod(shape), size=4000, replace=False)
    iz, iy, ix = np.unravel_index(flat, shape)
    Ms = M[:, iz, iy, ix][:, None, None, :, :]
    ref = _nt_entries(O.nr_computation(Ms, K[0]))[:, 0, 0, :]
    got = outs[0][:, iz, iy, ix]
    got = got[..., 0] + 1j * got[..., 1]
    np.testing.assert_allclose(got, ref, rtol=0, atol=3e-7 * max(np.abs(ref).max(), 1 / (4 * np.pi)))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("frame", [0, 1])
def test_polarization_from_nt(rsx, prec, frame):
    shape, c = (3, 16, 32), 3
    M = synth.morphology_random(shape, c, seed=55, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=56)
    nz, ny, nx = shape
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=2, frame=frame) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        p = torch.empty((3,) + shape + (2,), dtype=_tdt(prec), device="cuda")
        ctx.polarization(1, 0.8, p)
        got = p.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
    ref = O.polarization_from_nt(O.nr_computation(M, K[1]), O.e_field(0.8))
    if frame == 0:
        ref = O.rotate_back(ref, 0.8)
    scale = max(np.abs(ref).max(), 1 / (4 * np.pi))
    np.testing.assert_allclose(got, ref, rtol=0, atol=NT_TOL[prec] * scale)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("shape,c", [((4, 16, 16), 3), ((6, 32, 128), 4), ((1, 64, 64), 2),
                                     ((2, 8, 1024), 3), ((3, 256, 1024), 2), ((2, 512, 32), 2),
                                     ((3, 64, 512), 2), ((2, 512, 512), 3)])
def test_alg2_run_matches_oracle_and_alg1(rsx, shape, c, prec, where):
    M = synth.morphology_random(shape, c, seed=57, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=58)
    nz, ny, nx = shape
    angles = (0.0, 36.0, 180.0)
    ref = O.run_alg2(M, K, ENERGIES, VOXEL, angles_deg=angles)
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=2) as ctx:
        ctx.set_morphology(M if where == "host" else torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        got2 = ctx.run(angles)
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=1) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        got1 = ctx.run(angles)
    _close_img(got2, ref, prec)
    _close_img(got2, got1, prec)


def test_nt_refused_in_algorithm1_context(rsx):
    with rsx.Context(8, 8, 2, 2, VOXEL, precision=32) as ctx:
        ctx.set_morphology(synth.morphology_random((2, 8, 8), 2, seed=1))
        ctx.set_optical_constants([285.0], synth.optical_constants([285.0], 2, seed=2))
        out = torch.empty((5, 2, 8, 8, 2), device="cuda")
        with pytest.raises(rsx.RsxError) as e:
            ctx.nt(0, out)
        assert e.value.code == rsx.RSX_ERR_STATE


# ------------------------------------- linearity fast path (algorithm 3)
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("frame", [0, 1])
@pytest.mark.parametrize("shape,c", [((4, 16, 16), 3), ((6, 32, 128), 4), ((1, 64, 64), 2),
                                     ((5, 8, 32), 2), ((2, 1024, 8), 2), ((4, 1024, 64), 2),
                                     ((2, 512, 32), 2), ((4, 2048, 16), 2)])
def test_linear_path_matches_oracle_and_alg1(rsx, shape, c, prec, frame):
    M = synth.morphology_random(shape, c, seed=61, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=62)
    nz, ny, nx = shape
    angles = (0.0, 12.0, 180.0)
    mode = "literal" if frame == 0 else "lab"
    ref = O.run_linear(M, K, ENERGIES, VOXEL, angles_deg=angles, uT_mode=mode)
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=3, frame=frame) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        got3 = ctx.run(angles)
        img = torch.empty((ny, nx), dtype=_tdt(prec), device="cuda")
        ctx.scatter_angle(1, 0.4, img)
        one = img.cpu().numpy()
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=1, frame=frame) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(ENERGIES, K)
        got1 = ctx.run(angles)
        ctx.scatter_angle(1, 0.4, img)
        one1 = img.cpu().numpy()
    _close_img(got3, ref, prec)
    _close_img(got3, got1, prec)
    _close_img(one, one1, prec, r=1.5)


def test_linear_path_host_streamed_and_energy_subsets(rsx):
    shape, c = (4, 32, 64), 3
    E = list(np.linspace(270, 310, 5))
    M = synth.morphology_random(shape, c, seed=63)
    K = synth.optical_constants(E, c, seed=64)
    nz, ny, nx = shape
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=32, algorithm=3) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(E, K)
        full = ctx.run((0, 10, 180))
        part = ctx.run((0, 10, 180), energy_indices=[4, 1])
    np.testing.assert_array_equal(part, full[[4, 1]])
    ref = O.run_linear(M, K, E, VOXEL, angles_deg=(0, 10, 180), energy_indices=[0, 3])
    _close_img(full[[0, 3]], ref, 32)


@pytest.mark.parametrize("prec", [32, 64])
def test_linear_path_batched_angles_equal_angle_by_angle(rsx, prec):
    """The linearity path's run computes its angles in batches (images of a
    batch, then one rotate-and-accumulate pass); the step entry points one
    angle at a time must give the same average bit for bit, across more
    angles than one batch holds."""
    shape, c = (3, 32, 64), 3
    nz, ny, nx = shape
    M = synth.morphology_random(shape, c, seed=65, dtype=_real(prec))
    K = synth.optical_constants(ENERGIES, c, seed=66)
    start, inc, end = 0.0, 2.0, 180.0   # 91 angles
    n = rsx.angle_count(start, inc, end)
    with rsx.Context(nx, ny, nz, c, VOXEL, precision=prec, algorithm=3) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        got = ctx.run((start, inc, end), energy_indices=[1])
        img = torch.empty((ny, nx), dtype=_tdt(prec), device="cuda")
        acc = torch.zeros((ny, nx), dtype=_tdt(prec), device="cuda")
        for a in range(n):
            alpha = np.deg2rad(start + inc * a)
            ctx.scatter_angle(1, alpha, img)
            ctx.rotate_accumulate(img, alpha, acc)
        ref = (acc * (1.0 / n)).cpu().numpy()
    np.testing.assert_array_equal(got[0], ref)

