"""The allocation-free entry point rsx_scatter_angle_noalloc.

Some callers cannot allocate device memory (they run inside another
framework's memory pool, or on hosts that forbid cudaMalloc after start-up)
and so cannot create a context.  For them the library offers one entry point
whose working memory is a fixed array inside the library.  This file checks,
through the C ABI, that it gives the same image as the context path
(rsx_scatter_angle) and as the FP64 CPU oracle within the FP32 tolerance of
the parity tests, on two calls in a row (the second call must not be
disturbed by what the first left in the shared array), and that grids beyond
the fixed size are refused.

It is collected last on purpose, so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh
process.
"""
import numpy as np
import pytest

from paper_2209_13121_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_NORM_TOL = 1e-4   # relative L2 over pixels away from q = 0, as in the parity tests
FP32_PIX_TOL = 2e-3    # per pixel where X > 1e-4 max X


@pytest.fixture(scope="module")
def rsx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx as R
    return R


def _close(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    ny, nx = ref.shape
    iy, ix = np.meshgrid(np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    far = np.hypot(ix, iy) > 1.5
    rel = np.linalg.norm((got - ref)[far]) / np.linalg.norm(ref[far])
    assert rel <= FP32_NORM_TOL, rel
    big = ref > 1e-4 * ref.max()
    assert (np.abs(got - ref)[big] / ref[big]).max() <= FP32_PIX_TOL
    assert np.all(np.isfinite(got))


@pytest.mark.parametrize("frame", [0, 1])
def test_noalloc_matches_context_path_on_two_calls(rsx, frame):
    nz, ny, nx, c, dv = 12, 64, 128, 3, 5.0
    E = [280.0, 290.0]
    M = torch.from_numpy(synth.morphology_random((nz, ny, nx), c, seed=21)).cuda()
    K = synth.optical_constants(E, c, seed=22)
    with rsx.Context(nx, ny, nz, c, dv, precision=32, frame=frame) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants(E, K)
        for ie, alpha in ((0, 0.3), (1, 2.2)):          # two calls in a row
            out = torch.full((ny, nx), float("nan"), device="cuda")
            rsx.scatter_angle_noalloc(M, E[ie], K[ie], alpha, out, dv, frame=frame)
            ref = torch.empty((ny, nx), device="cuda")
            ctx.scatter_angle(ie, alpha, ref)
            torch.cuda.synchronize()
            _close(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_matches_the_oracle(rsx):
    """Directly against the FP64 CPU oracle on one small grid, in both
    frames, two calls in a row."""
    from oracle import cyrsoxs_oracle as O
    nz, ny, nx, c, dv = 6, 32, 64, 3, 5.0
    M = synth.morphology_random((nz, ny, nx), c, seed=31)
    K = synth.optical_constants([275.0, 300.0], c, seed=32)
    Md = torch.from_numpy(M).cuda()
    for frame, mode in ((0, "literal"), (1, "lab")):
        for ie, alpha in ((0, 0.5), (1, 1.9)):
            out = torch.full((ny, nx), float("nan"), device="cuda")
            rsx.scatter_angle_noalloc(Md, [275.0, 300.0][ie], K[ie], alpha, out, dv, frame=frame)
            torch.cuda.synchronize()
            ref = O.scatter_one_angle(M, K[ie], [275.0, 300.0][ie], dv, alpha, uT_mode=mode)
            _close(out.cpu().numpy(), ref)


def test_noalloc_second_grid_after_a_larger_one(rsx):
    """A smaller grid right after a larger one: nothing of the earlier call's
    scratch contents may show through."""
    dv = 5.0
    for (nz, ny, nx, c) in ((16, 128, 256, 2), (3, 16, 32, 4)):
        M = torch.from_numpy(synth.morphology_random((nz, ny, nx), c, seed=nz)).cuda()
        K = synth.optical_constants([285.0], c, seed=nx)
        out = torch.empty((ny, nx), device="cuda")
        rsx.scatter_angle_noalloc(M, 285.0, K[0], 0.7, out, dv)
        with rsx.Context(nx, ny, nz, c, dv, precision=32) as ctx:
            ctx.set_morphology(M)
            ctx.set_optical_constants([285.0], K)
            ref = torch.empty((ny, nx), device="cuda")
            ctx.scatter_angle(0, 0.7, ref)
            torch.cuda.synchronize()
        _close(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_refuses_grids_beyond_the_fixed_scratch(rsx):
    nz, ny, nx, c = 32, 256, 256, 1          # 2^21 voxels > 2^20
    M = torch.zeros((c, nz, ny, nx, 4), device="cuda")
    out = torch.empty((ny, nx), device="cuda")
    with pytest.raises(rsx.RsxError) as e:
        rsx.scatter_angle_noalloc(M, 285.0, np.zeros((c, 4)), 0.0, out, 5.0)
    assert e.value.code == rsx.RSX_ERR_INVALID
    assert "fixed scratch" in str(e.value)
