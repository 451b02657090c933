"""Line-grating validation (Sec. 5.2.2) against a trapezoid-stack Fourier
transform written from the mathematics.

A grating of trapezoidal lines (periodic along x, uniform along y, sloped
side walls in the x-z plane, vacuum above) is simulated at 17 keV with
1 nm voxels.  Its Bragg intensities are compared with

  * the stack of voxel rows the morphology actually holds: each row z is a
    rectangle [x_a, x_b) x [z, z+1), whose continuous transform is a
    product of two one-dimensional integrals.  The continuous transform of
    a voxelised body is its DFT times one voxel's transform, so
    |DFT|^2 = |F_stack|^2 / (sinc^2(q_x/2) sinc^2(q_z/2)) exactly; with the
    two q_z bins of the Ewald interpolation (the flat 17 keV sphere puts
    ~1e-3 of the weight on bin -1) the intensity ratios between orders must
    agree to rounding;
  * the smooth trapezoid (straight side walls), F = 4H [cos(q w_top/2) -
    cos(q w_bot/2)] / (q^2 (w_bot - w_top)) at q_z = 0, which the voxelised
    walls approximate (a few percent at the orders used).
"""
import math

import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O

NX, NY, NZ, P, H = 256, 4, 32, 64, 24
W_BOT, W_TOP = 40, 24
E_EV, DV = 17000.0, 1.0
ORDERS = [1, 2, 3, 4, 5, 6]


def _width(z):
    return int(round(W_BOT - (W_BOT - W_TOP) * (z + 0.5) / H))


def _row_span(z):
    w = _width(z)
    xa = P // 2 - w // 2
    return xa, xa + w


def grating_morphology(dtype=np.float64):
    M = np.zeros((2, NZ, NY, NX, 4), dtype=dtype)
    for z in range(H):
        xa, xb = _row_span(z)
        for c0 in range(0, NX, P):
            M[0, z, :, c0 + xa:c0 + xb, 0] = 1
    M[1, ..., 0] = 1 - M[0, ..., 0]
    return M


def constants():
    K = np.zeros((1, 2, 4))
    K[0, 0] = (2e-6, 1e-7, 2e-6, 1e-7)   # isotropic line material, hard X-ray scale
    return K


def _f_stack(qx, qz):
    """Continuous transform of one period's stack of voxel rows."""
    tot = 0j
    for z in range(H):
        xa, xb = _row_span(z)
        fx = (np.exp(-1j * qx * xb) - np.exp(-1j * qx * xa)) / (-1j * qx)
        fz = 1.0 if qz == 0 else (np.exp(-1j * qz * (z + 1)) - np.exp(-1j * qz * z)) / (-1j * qz)
        tot += fx * fz
    return tot


def _sinc(x):
    return 1.0 if x == 0 else math.sin(x) / x


def stack_intensity(m):
    """|DFT|^2 at Bragg order m (q_y = 0) with the two q_z bins and weights
    the Ewald sphere selects, times the polarisation factor (1 - r_x^2)."""
    qx = 2 * math.pi * m / (P * DV)
    k = 2 * math.pi * E_EV / 1239.84198
    qz = -k + math.sqrt(k * k - qx * qx)
    dqz = 2 * math.pi / (NZ * DV)
    t = qz / dqz
    z0 = math.floor(t)
    w = t - z0
    tot = 0.0
    for b, wt in ((z0, 1 - w), (z0 + 1, w)):
        qb = 2 * math.pi * b / (NZ * DV)
        tot += wt * abs(_f_stack(qx, qb)) ** 2 / (_sinc(qx / 2) ** 2 * _sinc(qb / 2) ** 2)
    rx = qx / k
    return tot * (1 - rx * rx)


def trapezoid_intensity(m):
    qx = 2 * math.pi * m / (P * DV)
    F = 4 * H * (math.cos(qx * W_TOP / 2) - math.cos(qx * W_BOT / 2)) / (qx * qx * (W_BOT - W_TOP))
    return F * F / _sinc(qx / 2) ** 2


def bragg_row(img):
    cy, cx = NY // 2, NX // 2
    return np.array([img[cy, cx + m * (NX // P)] for m in ORDERS])


def check_against_stack(img, rtol):
    sim = bragg_row(img)
    ana = np.array([stack_intensity(m) for m in ORDERS])
    np.testing.assert_allclose(sim / sim[0], ana / ana[0], rtol=rtol, atol=rtol * 1e-4)


def check_against_trapezoid(img):
    sim = bragg_row(img)
    ana = np.array([trapezoid_intensity(m) for m in ORDERS])
    for i in (2, 4):   # orders 3 and 5 (even orders vanish for the smooth shape)
        assert abs((sim[i] / sim[0]) / (ana[i] / ana[0]) - 1) < 0.05


def test_oracle_grating_matches_trapezoid_stack():
    img = O.run_alg1(grating_morphology(), constants(), [E_EV], DV, rotation=False)[0]
    check_against_stack(img, rtol=1e-9)


def test_oracle_grating_near_smooth_trapezoid():
    img = O.run_alg1(grating_morphology(), constants(), [E_EV], DV, rotation=False)[0]
    check_against_trapezoid(img)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,rtol", [(64, 1e-8), (32, 2e-3)])
def test_gpu_grating_matches_trapezoid_stack(prec, rtol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx
    M = grating_morphology(np.float32 if prec == 32 else np.float64)
    with rsx.Context(NX, NY, NZ, 2, DV, precision=prec) as ctx:
        ctx.set_morphology(M)
        ctx.set_optical_constants([E_EV], constants())
        img = ctx.run(rotation=False)[0]
    check_against_stack(img.astype(np.float64), rtol=rtol)
    check_against_trapezoid(img.astype(np.float64))
