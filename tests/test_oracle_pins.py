"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each case checks one oracle
function against a closed form, a brute-force sum, an exact invariant or a
validation statement of Sec. 5, chosen so that a dropped term, a wrong sign
or index, or a transposed operand in that function fails at least one case.
"""
import math
import os

import numpy as np
import pytest

from oracle import cyrsoxs_oracle as O
from paper_2209_13121_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FOUR_PI = 4.0 * math.pi


def _nt(dpar, bpar, dperp, bperp):
    return np.array([dpar, bpar, dperp, bperp], dtype=np.float64)


def _one_voxel(v, s, phi, theta):
    M = np.zeros((1, 1, 1, 1, 4))
    M[0, 0, 0, 0] = (v, s, phi, theta)
    return M


# ----------------------------------------------------------------- FFT (R9)
def test_fft_matches_brute_force_dft_odd_sizes():
    g = np.random.default_rng(1)
    Nz, Ny, Nx = 4, 5, 6
    p = g.standard_normal((3, Nz, Ny, Nx)) + 1j * g.standard_normal((3, Nz, Ny, Nx))
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    ref = np.zeros_like(p)
    for mz in range(Nz):
        for my in range(Ny):
            for mx in range(Nx):
                ph = np.exp(-2j * np.pi * (mz * z / Nz + my * y / Ny + mx * x / Nx))
                ref[:, mz, my, mx] = (p * ph[None]).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(O.fft3(p), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_fft_parseval_and_impulse():
    g = np.random.default_rng(2)
    p = g.standard_normal((3, 4, 8, 8)) + 1j * g.standard_normal((3, 4, 8, 8))
    pt = O.fft3(p)
    N = 4 * 8 * 8
    assert abs((np.abs(pt) ** 2).sum() - N * (np.abs(p) ** 2).sum()) < 1e-9 * N * (np.abs(p) ** 2).sum()
    imp = np.zeros((3, 4, 8, 8), complex)
    imp[:, 0, 0, 1] = 1.0  # impulse at x = 1 -> exp(-2 pi i m_x / 8)
    expect = np.exp(-2j * np.pi * np.arange(8) / 8)
    np.testing.assert_allclose(O.fft3(imp)[0, 2, 3, :], expect, atol=1e-14)


def test_q_axis_fft_order():
    q = O.q_axis(8, 5.0)
    dq = 2 * np.pi / (8 * 5.0)
    np.testing.assert_allclose(q, dq * np.array([0, 1, 2, 3, -4, -3, -2, -1]))


# ------------------------------------------------------- Eqs. ncorr, nrot
def test_director_closed_form_random_angles():
    """N_rot = R^T N_eff R equals a I + b d d^T with the director
    d = (cos phi sin theta, sin phi sin theta, cos theta), a = v (s n_perp +
    (1-s) t), b = v s (n_par - n_perp), t = Tr(N)/3 (uniaxial algebra)."""
    g = np.random.default_rng(3)
    n = 200
    v, s = g.random(n), g.random(n)
    phi, th = g.uniform(0, 2 * np.pi, n), g.uniform(0, np.pi, n)
    nt = _nt(3e-3, 1e-3, 1e-3, 4e-3)
    N = O.refractive_tensor(*nt)
    npar, nperp = 1 - nt[0] + 1j * nt[1], 1 - nt[2] + 1j * nt[3]
    t = (npar + 2 * nperp) / 3
    Nrot = O.rotated_tensor(O.effective_tensor(N, v, s), O.euler_R(phi, th))
    d = np.stack([np.cos(phi) * np.sin(th), np.sin(phi) * np.sin(th), np.cos(th)], axis=1)
    a = v * (s * nperp + (1 - s) * t)
    b = v * s * (npar - nperp)
    ref = a[:, None, None] * np.eye(3)[None] + b[:, None, None] * d[:, :, None] * d[:, None, :]
    np.testing.assert_allclose(Nrot, ref, atol=1e-14)


def test_euler_R_is_rotation():
    g = np.random.default_rng(4)
    R = O.euler_R(g.uniform(0, 7, 50), g.uniform(0, 4, 50))
    np.testing.assert_allclose(R @ np.transpose(R, (0, 2, 1)), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)


def test_polarization_closed_form_random_voxels():
    """p = sum_j [(a_j^2 - 1) e + (2 a_j b_j + b_j^2)(d_j . e) d_j] / (4 pi),
    which is (a I + b d d^T)^2 - I applied to e (d d^T is idempotent)."""
    g = np.random.default_rng(5)
    c, shape = 3, (2, 3, 4)
    M = synth.morphology_random(shape, c, seed=7, dtype=np.float64)
    nts = synth.optical_constants([285.0], c, seed=3, vacuum_last=False)[0]
    e = O.e_field(0.7)
    p = O.polarization(M, nts, e)
    ref = np.zeros((3,) + shape, complex)
    for j in range(c):
        npar, nperp = 1 - nts[j, 0] + 1j * nts[j, 1], 1 - nts[j, 2] + 1j * nts[j, 3]
        t = (npar + 2 * nperp) / 3
        v, s, phi, th = (M[j, ..., k] for k in range(4))
        a = v * (s * nperp + (1 - s) * t)
        b = v * s * (npar - nperp)
        d = np.stack([np.cos(phi) * np.sin(th), np.sin(phi) * np.sin(th), np.cos(th)])
        de = (d * e[:, None, None, None]).sum(axis=0)
        ref += ((a * a - 1)[None] * e[:, None, None, None] + ((2 * a * b + b * b) * de)[None] * d) / FOUR_PI
    np.testing.assert_allclose(p, ref, atol=1e-15)
    del g


def test_polarization_director_along_beam_sees_ordinary_index():
    """theta = 0: aligned axis along z, an in-plane e sees only n_perp,
    for every phi and every s."""
    nt = _nt(2e-3, 5e-4, 1e-3, 3e-3)
    nperp = 1 - nt[2] + 1j * nt[3]
    npar = 1 - nt[0] + 1j * nt[1]
    for phi in (0.0, 0.4, 2.0):
        p = O.polarization(_one_voxel(1.0, 1.0, phi, 0.0), nt[None], np.array([1.0, 0, 0]))
        np.testing.assert_allclose(p[:, 0, 0, 0], [(nperp ** 2 - 1) / FOUR_PI, 0, 0], atol=1e-16)
    # theta = pi/2, phi = 0: director along x, e = x sees n_par
    p = O.polarization(_one_voxel(1.0, 1.0, 0.0, np.pi / 2), nt[None], np.array([1.0, 0, 0]))
    np.testing.assert_allclose(p[:, 0, 0, 0], [(npar ** 2 - 1) / FOUR_PI, 0, 0], atol=1e-16)
    # theta = pi/2, phi = pi/2: director along y, e = y sees n_par, e = x sees n_perp
    p = O.polarization(_one_voxel(1.0, 1.0, np.pi / 2, np.pi / 2), nt[None], np.array([0, 1.0, 0]))
    np.testing.assert_allclose(p[:, 0, 0, 0], [0, (npar ** 2 - 1) / FOUR_PI, 0], atol=1e-16)
    p = O.polarization(_one_voxel(1.0, 1.0, np.pi / 2, np.pi / 2), nt[None], np.array([1.0, 0, 0]))
    np.testing.assert_allclose(p[:, 0, 0, 0], [(nperp ** 2 - 1) / FOUR_PI, 0, 0], atol=1e-16)


def test_polarization_unaligned_is_isotropic_trace_index():
    """s = 0: N_eff = v Tr(N)/3 I whatever phi, theta."""
    nt = _nt(2e-3, 5e-4, 1e-3, 3e-3)
    t = ((1 - nt[0] + 1j * nt[1]) + 2 * (1 - nt[2] + 1j * nt[3])) / 3
    for phi, th in ((0.3, 1.1), (5.0, 2.9)):
        for v in (1.0, 0.6):
            e = O.e_field(0.9)
            p = O.polarization(_one_voxel(v, 0.0, phi, th), nt[None], e)
            np.testing.assert_allclose(p[:, 0, 0, 0], ((v * t) ** 2 - 1) / FOUR_PI * e, atol=1e-16)


def test_polarization_vacuum_component_subtracts_identity():
    """Reading R3: a component with v = 0 still contributes -e / (4 pi)."""
    nt = _nt(2e-3, 5e-4, 1e-3, 3e-3)
    e = O.e_field(0.3)
    p = O.polarization(_one_voxel(0.0, 0.5, 1.0, 1.0), nt[None], e)
    np.testing.assert_allclose(p[:, 0, 0, 0], -e / FOUR_PI, atol=1e-16)


def test_polarization_tensor_is_complex_symmetric_and_linear():
    """N_t = sum_j (N_rot^j N_rot^j - I)/(4 pi) is complex symmetric (Sec. 4.3)
    and p is linear in e."""
    M = synth.morphology_random((1, 2, 3), 2, seed=11, dtype=np.float64)
    nts = synth.optical_constants([284.0], 2, seed=5, vacuum_last=False)[0]
    cols = [O.polarization(M, nts, np.eye(3)[k]).reshape(3, -1) for k in range(3)]
    Nt = np.stack(cols, axis=1)  # Nt[a, b, voxel]
    np.testing.assert_allclose(Nt, np.transpose(Nt, (1, 0, 2)), atol=1e-16)
    e = np.array([0.3, -0.7, 0.2])
    p = O.polarization(M, nts, e).reshape(3, -1)
    np.testing.assert_allclose(p, np.einsum("abv,b->av", Nt, e), atol=1e-16)


def test_rotate_back_undoes_e_rotation_for_isotropic_material():
    """U^T U (1,0,0) = (1,0,0): an isotropic voxel gives U^T p = chi x-hat."""
    nt = _nt(2e-3, 5e-4, 2e-3, 5e-4)  # n_par = n_perp: isotropic
    for alpha in (0.0, 0.5, 2.0):
        p = O.rotate_back(O.polarization(_one_voxel(1, 1, 0.3, 0.8), nt[None], O.e_field(alpha)), alpha)
        n = 1 - nt[0] + 1j * nt[1]
        np.testing.assert_allclose(p[:, 0, 0, 0], [(n * n - 1) / FOUR_PI, 0, 0], atol=1e-16)


# ------------------------------------------------------ Eqs. 3Dscatter, Ewald
def _sphere_rhat(E, qx, qy):
    k = O.wavenumber(E)
    qz_plus_k = np.sqrt(k * k - qx * qx - qy * qy)
    return np.stack([qx / k, qy / k, qz_plus_k / k]), k


def test_ewald_constant_field_closed_form():
    """p~ = chi e for every q (a point scatterer): X = k^4 |chi|^2 (1 - (r.e)^2)
    with r on the Ewald sphere, independent of the q_z interpolation."""
    E, dv = 285.0, 5.0
    Nz, Ny, Nx = 4, 8, 6
    chi = 0.3 - 0.2j
    for e in (np.array([1.0, 0, 0]), O.e_field(0.6)):
        pt = np.broadcast_to((chi * e)[:, None, None, None], (3, Nz, Ny, Nx)).copy()
        X = O.ewald(pt, E, dv)
        qx = O.q_axis(Nx, dv)[None, :]
        qy = O.q_axis(Ny, dv)[:, None]
        r, k = _sphere_rhat(E, *np.broadcast_arrays(qx, qy))
        re = (r * e[:, None, None]).sum(axis=0)
        np.testing.assert_allclose(X, k ** 4 * abs(chi) ** 2 * (1 - re ** 2), rtol=1e-12)


def test_ewald_zero_outside_sphere():
    """Pixels with q_perp > k have no real q_z and read zero (Eq. Ewald)."""
    E, dv = 120.0, 2.0  # k = 0.608 nm^-1, Nyquist q = 1.57 nm^-1
    pt = np.ones((3, 2, 16, 16), complex)
    X = O.ewald(pt, E, dv)
    qx = O.q_axis(16, dv)[None, :]
    qy = O.q_axis(16, dv)[:, None]
    outside = qx ** 2 + qy ** 2 > O.wavenumber(E) ** 2
    assert outside.sum() > 20
    assert np.all(X[outside] == 0.0) and np.all(X[~outside] > 0.0)


def test_ewald_tent_weight_for_z_uniform_stack():
    """A morphology uniform along z has p~ only in the q_z = 0 plane, with
    p~ = Nz P2(q_x, q_y).  Linear interpolation between the bracketing bins
    then gives X_3D = max(0, 1 - |q_z|/dq_z) Nz^2 X_2D, where X_2D is the
    Nz = 1 image (whose single plane is always used)."""
    E, dv = 285.0, 5.0
    Nz, Ny, Nx = 16, 16, 16
    M2 = synth.morphology_random((1, Ny, Nx), 2, seed=21, dtype=np.float64)
    M3 = np.repeat(M2, Nz, axis=1)
    nts = synth.optical_constants([E], 2, seed=9)[0]
    X2 = O.fftshift2(O.ewald(O.fft3(O.polarization(M2, nts, np.array([1.0, 0, 0]))), E, dv))
    X3 = O.fftshift2(O.ewald(O.fft3(O.polarization(M3, nts, np.array([1.0, 0, 0]))), E, dv))
    k = O.wavenumber(E)
    qx = np.fft.fftshift(O.q_axis(Nx, dv))[None, :]
    qy = np.fft.fftshift(O.q_axis(Ny, dv))[:, None]
    qz = -k + np.sqrt(k * k - qx * qx - qy * qy)
    dqz = 2 * np.pi / (Nz * dv)
    tent = np.maximum(0.0, 1.0 - np.abs(qz) / dqz)
    assert (tent > 0).sum() > 10 and (tent == 0).sum() > 10  # both regimes present
    np.testing.assert_allclose(X3, tent * Nz ** 2 * X2, rtol=1e-9, atol=1e-12 * X3.max())


def test_point_scatterer_full_pipeline():
    """One isotropic voxel (plus vacuum elsewhere): away from q = 0 the image
    is k^4 |chi|^2 (1 - r_x^2) with chi = (n^2 - 1)/(4 pi) at alpha = 0."""
    E, dv = 285.0, 5.0
    shape = (4, 8, 8)
    M = np.zeros((2,) + shape + (4,))
    M[0, 1, 2, 3, 0] = 1.0
    M[1, ..., 0] = 1.0
    M[1, 1, 2, 3, 0] = 0.0
    nts = np.zeros((2, 4))
    nts[0] = (1e-3, 2e-3, 1e-3, 2e-3)
    X = O.ewald(O.fft3(O.polarization(M, nts, np.array([1.0, 0, 0]))), E, dv)
    n = 1 - 1e-3 + 2e-3j
    chi_contrast = (n * n - 1) / FOUR_PI  # vacuum voxels contribute 0 contrast
    qx = O.q_axis(8, dv)[None, :]
    qy = O.q_axis(8, dv)[:, None]
    r, k = _sphere_rhat(E, *np.broadcast_arrays(qx, qy))
    ref = k ** 4 * abs(chi_contrast) ** 2 * (1 - r[0] ** 2)
    mask = np.ones_like(ref, bool)
    mask[0, 0] = False
    np.testing.assert_allclose(X[mask], ref[mask], rtol=1e-10)


# -------------------------------------------------- detector rotation (R6)
def test_rotate_image_identity_and_quarter_turn():
    g = np.random.default_rng(8)
    img = g.random((8, 8))
    np.testing.assert_array_equal(O.rotate_image(img, 0.0), img)
    out = O.rotate_image(img, np.pi / 2)
    c = 4
    ref = np.zeros_like(img)
    for iy in range(8):
        for ix in range(8):
            sx, sy = c - (iy - c), c + (ix - c)  # U(90) (Qx, Qy) = (-Qy, Qx)
            if 0 <= sx < 8 and 0 <= sy < 8:
                ref[iy, ix] = img[sy, sx]
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_rotate_image_reproduces_linear_field():
    """Bilinear sampling is exact on a linear function (interior pixels)."""
    Ny, Nx = 12, 16
    iy, ix = np.meshgrid(np.arange(Ny, dtype=float), np.arange(Nx, dtype=float), indexing="ij")
    img = 0.5 + 0.25 * ix - 0.125 * iy
    a = 0.3
    out = O.rotate_image(img, a)
    cx, cy = Nx // 2, Ny // 2
    fx = cx + math.cos(a) * (ix - cx) - math.sin(a) * (Nx / Ny) * (iy - cy)
    fy = cy + math.sin(a) * (Ny / Nx) * (ix - cx) + math.cos(a) * (iy - cy)
    inside = (fx >= 0) & (fx <= Nx - 1) & (fy >= 0) & (fy <= Ny - 1)
    np.testing.assert_allclose(out[inside], (0.5 + 0.25 * fx - 0.125 * fy)[inside], atol=1e-12)


def test_angle_list_inclusive():
    assert len(O.angle_list(0, 2, 180)) == 91
    assert len(O.angle_list(0, 30, 180)) == 7
    assert len(O.angle_list(0, 7, 20)) == 3
    np.testing.assert_array_equal(O.angle_list(0, 2, 180, rotation=False), [0.0])


# ----------------------------------------------- Algorithm 1 / Sec. 5 physics
def test_polydomain_quarter_turn_equals_rotated_sample():
    """Sec. 3.3: averaging over e rotations simulates copies of the model
    rotated about z.  With the frame-consistent reading, the image for the
    single angle 90 deg equals the e = x image of the model turned by -90 deg
    (isotropic materials; the grid turn is exact on a square grid)."""
    E, dv, N = 285.0, 5.0, 16
    M = synth.morphology_random((2, N, N), 3, seed=31, binary=True, dtype=np.float64)
    M[..., 1] = 0.0  # unaligned -> isotropic
    nts = synth.optical_constants([E], 3, seed=4)
    out = O.run_alg1(M, nts, [E], dv, angles_deg=(90.0, 1.0, 90.0), uT_mode="lab")[0]
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Mt = M[:, :, xx, (-yy) % N]          # new(x, y) = old(-y, x)
    ref = O.run_alg1(Mt, nts, [E], dv, rotation=False, uT_mode="lab")[0]
    mask = np.ones((N, N), bool)
    mask[0, :] = mask[:, 0] = False        # Nyquist row/column leave the grid
    mask[N // 2, N // 2] = False           # q = 0
    np.testing.assert_allclose(out[mask], ref[mask], rtol=1e-9, atol=1e-12 * ref[mask].max())


def test_isotropic_prerotation_image_independent_of_angle_literal():
    """Reading R5 (literal): for isotropic materials U^T p = chi x-hat, so the
    image before the detector rotation is the same for every angle."""
    E, dv = 290.0, 5.0
    M = synth.morphology_random((2, 8, 8), 2, seed=12, dtype=np.float64)
    M[..., 1] = 0.0
    nts = synth.optical_constants([E], 2, seed=2)[0]
    ref = O.scatter_one_angle(M, nts, E, dv, 0.0)
    for a in (0.4, 1.3, 2.5):
        np.testing.assert_allclose(O.scatter_one_angle(M, nts, E, dv, a), ref, rtol=1e-10, atol=1e-14 * ref.max())


def test_literal_and_lab_agree_paraxially():
    """Reading R5: at 17 keV (Sec. 5.2.2) r-hat is z to O(q/k) and the literal
    and frame-consistent readings agree to O((q/k)^2)."""
    E, dv = 17000.0, 1.0
    M = synth.morphology_random((2, 16, 16), 3, seed=13, dtype=np.float64)
    nts = synth.optical_constants([E], 3, seed=6)
    a = O.run_alg1(M, nts, [E], dv, angles_deg=(0, 45, 90), uT_mode="literal")[0]
    b = O.run_alg1(M, nts, [E], dv, angles_deg=(0, 45, 90), uT_mode="lab")[0]
    qmax = np.pi / dv * np.sqrt(2)
    ratio = (qmax / O.wavenumber(E)) ** 2
    assert np.abs(a - b).max() <= 4 * ratio * np.abs(b).max()


def _quarter_turn(M):
    """The model turned by -90 deg about z: new(x, y) = old(-y, x) on the
    periodic grid, and every director's azimuth phi turned by -90 deg."""
    N = M.shape[2]
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    Mt = M[:, :, xx, (-yy) % N].copy()
    Mt[..., 2] -= np.pi / 2
    return Mt


def test_polydomain_average_equals_rotated_copies_anisotropic():
    """Sec. 3.3: the e-rotation average equals the average of copies of the
    model turned about z, each seen with e = x (frame-consistent reading,
    anisotropic materials with random directors, angles 0:90:270)."""
    E, dv, N = 285.0, 5.0, 16
    M = synth.morphology_random((2, N, N), 3, seed=14, dtype=np.float64)
    nts = synth.optical_constants([E], 3, seed=7)
    avg = O.run_alg1(M, nts, [E], dv, angles_deg=(0, 90, 270), uT_mode="lab")[0]
    copies = np.zeros_like(avg)
    Mk = M
    for _ in range(4):
        copies += O.run_alg1(Mk, nts, [E], dv, rotation=False, uT_mode="lab")[0]
        Mk = _quarter_turn(Mk)
    copies /= 4
    mask = np.ones((N, N), bool)
    mask[0, :] = mask[:, 0] = False
    mask[N // 2, N // 2] = False
    np.testing.assert_allclose(avg[mask], copies[mask], rtol=1e-9, atol=1e-12 * copies[mask].max())


def test_rotation_zero_angle_equals_rotation_off():
    E, dv = 285.0, 5.0
    M = synth.morphology_random((2, 8, 8), 2, seed=15, dtype=np.float64)
    nts = synth.optical_constants([E], 2, seed=8)
    a = O.run_alg1(M, nts, [E], dv, angles_deg=(0, 5, 0))
    b = O.run_alg1(M, nts, [E], dv, rotation=False)
    np.testing.assert_array_equal(a, b)


def test_energy_subsets_are_rows_of_full_run():
    E = [270.0, 285.0, 300.0]
    M = synth.morphology_random((1, 8, 8), 2, seed=16, dtype=np.float64)
    nts = synth.optical_constants(E, 2, seed=1)
    full = O.run_alg1(M, nts, E, 5.0, angles_deg=(0, 60, 120))
    part = O.run_alg1(M, nts, E, 5.0, angles_deg=(0, 60, 120), energy_indices=[2, 0])
    np.testing.assert_array_equal(part, full[[2, 0]])


def _isi(E, dd, db):
    """ISI of a binary isotropic 2-D pattern at one energy."""
    N, dv = 32, 5.0
    M = synth.morphology_disk((1, N, N), 6.0)
    nts = np.zeros((1, 2, 4))
    nts[0, 0] = (dd, db, dd, db)
    img = O.run_alg1(M, nts, [E], dv, rotation=False)[0]
    img[N // 2, N // 2] = 0.0
    return img.sum()


def test_integrated_intensity_energy_law():
    """Sec. 5.1.1: the integrated scattering intensity scales as
    (d_delta^2 + d_beta^2) E^4 (to first order in delta, beta, and up to the
    polarisation factor 1 - r_x^2, which changes by < 1% between the two
    energies here)."""
    r1 = _isi(270.0, 1e-3, 2e-4)
    r2 = _isi(310.0, 4e-4, 1e-3)
    law = (270.0 / 310.0) ** 4 * (1e-6 + 4e-8) / (1.6e-7 + 1e-6)
    assert abs(r1 / r2 / law - 1) < 0.01


def test_sphere_form_factor():
    """Sec. 5.1.2: azimuthal average of a 3-D sphere's pattern follows
    [3 (sin qr - qr cos qr)/(qr)^3]^2 (Eq. FoamFactor) up to discretisation,
    normalised at the lowest q bin, tested below the first minimum."""
    N, Nz, dv, R = 64, 32, 5.0, 6.0
    M = synth.morphology_sphere((Nz, N, N), R)
    nts = np.zeros((1, 2, 4))
    nts[0, 0] = (1e-3, 5e-4, 1e-3, 5e-4)
    E = 2000.0  # flat Ewald sphere over the tested range
    img = O.run_alg1(M, nts, [E], dv, rotation=False)[0]
    dq = 2 * np.pi / (N * dv)
    iy, ix = np.meshgrid(np.arange(N) - N // 2, np.arange(N) - N // 2, indexing="ij")
    qr = np.hypot(ix, iy) * dq
    r_nm = R * dv
    bins = np.arange(1, 9)
    sim, ana = [], []
    for b in bins:
        sel = np.abs(qr / dq - b) < 0.5
        sim.append(img[sel].mean())
        x = qr[sel] * r_nm
        ana.append((((np.sin(x) - x * np.cos(x)) / x ** 3) ** 2).mean())
    sim = np.array(sim) / sim[0]
    ana = np.array(ana) / ana[0]
    first_min = 4.493 / r_nm
    keep = bins * dq < 0.85 * first_min
    assert keep.sum() >= 4
    np.testing.assert_allclose(sim[keep], ana[keep], rtol=0.08)


def test_disk_projection_airy():
    """A z-uniform disk (Nz = 1) scatters as the 2-D disk transform
    [2 J1(qR)/(qR)]^2; checked below the first zero as for the sphere."""
    from scipy.special import j1
    N, dv, R = 128, 5.0, 10.0
    M = synth.morphology_disk((1, N, N), R)
    nts = np.zeros((1, 2, 4))
    nts[0, 0] = (1e-3, 5e-4, 1e-3, 5e-4)
    img = O.run_alg1(M, nts, [5000.0], dv, rotation=False)[0]
    dq = 2 * np.pi / (N * dv)
    iy, ix = np.meshgrid(np.arange(N) - N // 2, np.arange(N) - N // 2, indexing="ij")
    qr = np.hypot(ix, iy) * dq
    r_nm = R * dv
    sim, ana = [], []
    bins = np.arange(1, 8)
    for b in bins:
        sel = np.abs(qr / dq - b) < 0.5
        sim.append(img[sel].mean())
        x = qr[sel] * r_nm
        ana.append(((2 * j1(x) / x) ** 2).mean())
    sim, ana = np.array(sim) / sim[0], np.array(ana) / ana[0]
    keep = bins * dq < 0.85 * 3.8317 / r_nm
    assert keep.sum() >= 4
    np.testing.assert_allclose(sim[keep], ana[keep], rtol=0.08)


def test_square_wave_grating_odd_harmonics():
    """Sec. 5.2.2 geometry (lines along y, 50% duty): the q_y = 0 row has
    intensity only at odd multiples of the grating frequency."""
    N, period = 64, 8
    M = synth.morphology_grating((1, N, N), period, period // 2, axis="x")
    nts = np.zeros((1, 2, 4))
    nts[0, 0] = (1e-3, 5e-4, 1e-3, 5e-4)
    img = O.run_alg1(M, nts, [17000.0], 1.0, rotation=False)[0]
    row = img[N // 2]
    m = np.arange(N) - N // 2
    fund = N // period
    odd = (m % fund == 0) & ((m // fund) % 2 == 1)
    other = ~odd & (m != 0)
    assert row[odd].min() > 1e6 * max(row[other].max(), 1e-300)
    assert np.all(img[np.arange(N) != N // 2][:, m != 0].max() <= 1e-12 * row.max())


def test_hexagonal_lattice_bragg_positions():
    """Sec. 5.2.1: circles on a hexagonal lattice give Bragg peaks at
    q*, sqrt(3) q*, sqrt(4) q*, sqrt(7) q*, ... (tests/golden fixture).
    Lattice constant a = 30 voxels, box 4a x 2 a sqrt(3) (104 voxels, 0.08
    voxel from commensurate), so every reciprocal vector lands on a pixel."""
    ratios = np.loadtxt(os.path.join(GOLDEN, "hex_lattice_peak_ratios.txt"))
    a_vox, Nx, Ny, dv = 30.0, 120, 104, 1.0
    M = synth.morphology_hex_lattice((1, Ny, Nx), a_vox, 3.0)
    nts = np.zeros((1, 2, 4))
    nts[0, 0] = (1e-3, 5e-4, 1e-3, 5e-4)
    img = O.run_alg1(M, nts, [20000.0], dv, rotation=False)[0]
    img[Ny // 2, Nx // 2] = 0.0
    qx = np.fft.fftshift(O.q_axis(Nx, dv))[None, :]
    qy = np.fft.fftshift(O.q_axis(Ny, dv))[:, None]
    q = np.hypot(qx, qy) * np.ones_like(img)
    qstar = 4 * np.pi / (np.sqrt(3) * a_vox * dv)
    dq = 2 * np.pi / (Ny * dv)
    inrange = q < (ratios.max() + 0.2) * qstar
    vals = np.where(inrange, img, 0.0)
    # the 36 brightest pixels in range sit on the predicted rings
    order = np.argsort(vals.ravel())[::-1][:36]
    for val in q.ravel()[order] / qstar:
        assert np.min(np.abs(val - ratios)) * qstar < 1.2 * dq
    # every predicted ring holds a peak far above the background (the
    # median pixel in range: Bragg peaks occupy a few dozen of ~7000 pixels)
    bg = np.median(img[inrange & (q > 0.5 * qstar)])
    for rr in ratios:
        ring = np.abs(q - rr * qstar) < 1.2 * dq
        assert img[ring].max() > 1e3 * bg


# ------------------------------------------------------ Algorithms 2 and 3
def test_nr_computation_closed_form_and_symmetry():
    """Algorithm 3's N_t equals sum_j [(a_j^2 - 1) I + (2 a_j b_j + b_j^2) d_j d_j^T]
    / (4 pi) (uniaxial algebra) and is complex symmetric (Sec. 4.3)."""
    c, shape = 3, (2, 3, 4)
    M = synth.morphology_random(shape, c, seed=41, dtype=np.float64)
    nts = synth.optical_constants([287.0], c, seed=42, vacuum_last=False)[0]
    Nt = O.nr_computation(M, nts)
    ref = np.zeros(shape + (3, 3), complex)
    for j in range(c):
        npar, nperp = 1 - nts[j, 0] + 1j * nts[j, 1], 1 - nts[j, 2] + 1j * nts[j, 3]
        t = (npar + 2 * nperp) / 3
        v, s, phi, th = (M[j, ..., k] for k in range(4))
        a = v * (s * nperp + (1 - s) * t)
        b = v * s * (npar - nperp)
        d = np.stack([np.cos(phi) * np.sin(th), np.sin(phi) * np.sin(th), np.cos(th)], axis=-1)
        ref += ((a * a - 1)[..., None, None] * np.eye(3)
                + (2 * a * b + b * b)[..., None, None] * d[..., :, None] * d[..., None, :]) / FOUR_PI
    np.testing.assert_allclose(Nt, ref, atol=1e-15)
    np.testing.assert_allclose(Nt, np.swapaxes(Nt, -1, -2), atol=1e-16)


def test_algorithm2_equals_algorithm1():
    """Sec. 4.3: Algorithm 2 reorganises Algorithm 1 (N_t precomputed per
    energy); the images agree up to rounding, in both frames."""
    E = [275.0, 290.0]
    M = synth.morphology_random((3, 8, 16), 3, seed=43, dtype=np.float64)
    K = synth.optical_constants(E, 3, seed=44)
    for mode in ("literal", "lab"):
        a1 = O.run_alg1(M, K, E, 5.0, angles_deg=(0, 40, 160), uT_mode=mode)
        a2 = O.run_alg2(M, K, E, 5.0, angles_deg=(0, 40, 160), uT_mode=mode)
        np.testing.assert_allclose(a2, a1, rtol=1e-10, atol=1e-14 * a1.max())


def test_linearity_restatement_equals_algorithm1():
    """p~ is linear in e and the FFT is linear: forming FFT(N_t x) and
    FFT(N_t y) once per energy gives Algorithm 1's images up to rounding."""
    E = [278.0, 295.0]
    M = synth.morphology_random((4, 8, 16), 3, seed=45, dtype=np.float64)
    K = synth.optical_constants(E, 3, seed=46)
    for mode in ("literal", "lab"):
        a1 = O.run_alg1(M, K, E, 5.0, angles_deg=(0, 20, 180), uT_mode=mode)
        al = O.run_linear(M, K, E, 5.0, angles_deg=(0, 20, 180), uT_mode=mode)
        np.testing.assert_allclose(al, a1, rtol=1e-10, atol=1e-14 * a1.max())


# ------------------------------------- sampled pixels of sparse morphologies
def test_dft_sparse_is_the_dft():
    g = np.random.default_rng(31)
    shape = (5, 6, 8)
    iz, iy, ix = (g.integers(0, n, 7) for n in shape)
    vals = g.normal(size=(3, 7)) + 1j * g.normal(size=(3, 7))
    dense = np.zeros((3,) + shape, complex)
    np.add.at(dense, (slice(None), iz, iy, ix), vals)
    ref = np.fft.fftn(dense, axes=(1, 2, 3))
    kz, ky, kx = (g.integers(0, n, 11) for n in shape)
    np.testing.assert_allclose(O.dft_sparse(vals, iz, iy, ix, shape, kz, ky, kx),
                               ref[:, kz, ky, kx], rtol=0, atol=1e-12)


def test_ewald_pixels_equals_ewald():
    g = np.random.default_rng(32)
    shape = (4, 8, 16)
    pt = g.normal(size=(3,) + shape) + 1j * g.normal(size=(3,) + shape)
    for E, dv in ((285.0, 5.0), (270.0, 2.0)):   # 2 nm: corners off the sphere
        full = O.ewald(pt, E, dv)
        iy, ix = np.meshgrid(np.arange(8), np.arange(16), indexing="ij")
        got = O.ewald_pixels(lambda b, y, x: pt[:, b, y, x], E, dv, shape, iy.ravel(), ix.ravel())
        np.testing.assert_allclose(got.reshape(8, 16), full, rtol=1e-13, atol=0)


def test_sparse_pixels_equal_the_full_path():
    """Linearity of the DFT: the sampled path for a vacuum-plus-sparse
    morphology equals Algorithm 1's full image (both frames)."""
    from paper_2209_13121_gb300 import synth
    shape, c = (6, 16, 32), 3
    sp = synth.sparse_voxels(shape, c, 40, seed=33)
    M = synth.morphology_sparse(shape, c, sp)
    K = synth.optical_constants([285.0], c, seed=34)
    iy, ix = np.meshgrid(np.arange(16), np.arange(32), indexing="ij")
    for mode in ("literal", "lab"):
        full = O.scatter_one_angle(M, K[0], 285.0, 5.0, 0.7, uT_mode=mode)
        got = O.scatter_sparse_pixels(sp, shape, K[0], 285.0, 5.0, 0.7, iy.ravel(), ix.ravel(),
                                      uT_mode=mode).reshape(16, 32)
        np.testing.assert_allclose(O.fftshift2(got), full, rtol=0, atol=1e-13 * full.max())


def test_rotate_sampled_equals_the_full_rotation():
    """The detector rotation read at selected output pixels equals the full
    rotated image there (R6), on square and non-square grids, for angles
    that land between pixels and at exact quarter turns, including output
    pixels whose source corners leave the grid."""
    g = np.random.default_rng(35)
    for shape in ((16, 16), (12, 20), (9, 7)):
        img = g.random(shape)
        iy, ix = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
        for a in (0.0, 0.3, math.pi / 2, 2.9, -1.2):
            full = O.rotate_image(img, a)
            got = O.rotate_sampled(lambda sy, sx: img[sy, sx], shape, a, iy.ravel(), ix.ravel())
            np.testing.assert_allclose(got.reshape(shape), full, rtol=0, atol=1e-14)


def test_run_alg1_sparse_pixels_equal_the_full_path():
    """Algorithm 1's average at sampled pixels of a vacuum-plus-sparse
    morphology equals run_alg1's full image (both frames, rotation on and
    off, a ragged angle list)."""
    from paper_2209_13121_gb300 import synth
    shape, c, E = (4, 16, 24), 3, 290.0
    sp = synth.sparse_voxels(shape, c, 30, seed=36)
    M = synth.morphology_sparse(shape, c, sp)
    K = synth.optical_constants([E], c, seed=37)
    oy, ox = np.meshgrid(np.arange(16), np.arange(24), indexing="ij")
    for mode in ("literal", "lab"):
        for rot in (True, False):
            full = O.run_alg1(M, K, [E], 5.0, angles_deg=(10.0, 35.0, 150.0), rotation=rot,
                              uT_mode=mode)[0]
            got = O.run_alg1_sparse_pixels(sp, shape, K[0], E, 5.0, (10.0, 35.0, 150.0),
                                           oy.ravel(), ox.ravel(), rotation=rot,
                                           uT_mode=mode).reshape(16, 24)
            np.testing.assert_allclose(got, full, rtol=0, atol=1e-13 * full.max())
