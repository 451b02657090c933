"""FP64 CPU oracle of the P-RSoXS forward model (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
restatement of the method that the CUDA path is checked against.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import
it; the library never does, and it shares no code with the library.

Every step follows the paper in its own order and notation:

  Sec. 3.3 step 1  effective refractive tensor        Eq. (ncorr)
  Sec. 3.3 step 2  rotated tensor, R = B C D          Eqs. (rotBCD), (nrot)
  Sec. 3.3 step 3  induced polarisation               Eq. (polarization)
                   rotation of e and p <- U^T p       Sec. 3.3, Algorithm 1
  Sec. 3.3 step 4  FFT of p                            (numpy's FFT as a step)
  Sec. 3.3 step 5  scatter                             Eq. (3Dscatter)
  Sec. 3.3 step 6  Ewald projection + interpolation    Eq. (Ewald)
  Sec. 4           detector rotation and average      Algorithm 1
  Sec. 4.3         N_t per energy, p = N_t . e         Algorithms 2 and 3
  linearity        p~(alpha) from FFTs of N_t's columns  (exact restatement
                   of Algorithm 2: e(alpha) = cos a x + sin a y, FFT linear)

Readings of points the paper leaves open (the design notes list the same):

  R1  n = 1 - delta + i beta along each principal axis.
  R2  "N_rot : N_rot" in Eq. (polarization) is the matrix product.
  R3  The identity is subtracted once per component, as written.
  R4  The extraordinary axis of the uniaxial tensor lies on the initial
      alignment axis (0,0,1); R = B C D with passive rotations D (phi about
      Z), C (theta about Y), B (psi = 0 about Z), so the director is
      d = R^T z = (cos phi sin theta, sin phi sin theta, cos theta).
  R5  p <- U^T p is applied to the components of p; the grid and r-hat stay
      in the material frame ("literal").  uT_mode="lab" skips it, which
      is the frame-consistent alternative (norm-preserving).
  R6  The detector image (in fftshift order) is rotated about q = 0 by
      sampling the image at U(alpha) Q with bilinear interpolation, zero
      outside the grid, then averaged over the angles.
  R7  The angle list start:increment:end includes end when (end-start)/inc
      is an integer (to 1e-6).
  R8  X is interpolated linearly between the two bracketing integer q_z bins
      (periodic wrap), each bin's |Y|^2 taken with r-hat at the exact k_out.
  R9  FFT: forward sign exp(-i ...), unnormalised.
  R10 The detector uses the FFT's (q_x, q_y) grid; pixels with
      q_x^2 + q_y^2 > k^2 are zero.
  R11 Within a component, voxels are ordered x fastest, then y, then z.
  R12 lambda = hc / E with hc = 1239.84198 eV nm.

Pins: tests/test_oracle_pins.py checks every function here against closed
forms, brute force and invariants.  Parity unpinned: the sign of the
imaginary part in R1 (complex conjugation leaves every validation quantity
of Sec. 5 unchanged), the 1/(4 pi) placement and the absolute intensity
scale (Sec. 5.1 compares shapes and relative scaling only).
"""
from __future__ import annotations

import math

import numpy as np

HC_EV_NM = 1239.84198  # R12


# ---------------------------------------------------------------- Sec. 3.2
def wavelength_nm(E_eV: float) -> float:
    return HC_EV_NM / E_eV


def wavenumber(E_eV: float) -> float:
    """|k_in| = 2 pi / lambda in nm^-1."""
    return 2.0 * math.pi / wavelength_nm(E_eV)


def refractive_tensor(delta_par, beta_par, delta_perp, beta_perp) -> np.ndarray:
    """Uniaxial refractive tensor N (Eq. uniaxialRefrativeIndex), complex 3x3.

    The paper writes diag(n_par, n_perp, n_perp); per reading R4 the
    extraordinary value n_par sits on the initial alignment axis z, so in
    x, y, z order the diagonal is (n_perp, n_perp, n_par).  R1 gives the
    complex values.
    """
    n_par = 1.0 - delta_par + 1j * beta_par
    n_perp = 1.0 - delta_perp + 1j * beta_perp
    return np.diag(np.array([n_perp, n_perp, n_par], dtype=np.complex128))


# ---------------------------------------------------------------- Sec. 3.3
def effective_tensor(N: np.ndarray, v: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Eq. (ncorr): N_eff = v (s N + (1 - s) (1/3) Tr(N) I), per voxel.

    v, s: arrays of shape (n,).  Returns (n, 3, 3) complex."""
    iso = np.trace(N) / 3.0 * np.eye(3)
    return v[:, None, None] * (s[:, None, None] * N[None] + (1.0 - s)[:, None, None] * iso[None])


def euler_R(phi: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Eq. (rotBCD): R = B C D, per voxel, (n, 3, 3) real.

    D: rotation by phi about Z, C: rotation by theta about Y, B: rotation by
    psi about Z with psi = 0 (a uniaxial component has no third angle, Sec.
    3.1).  Passive (frame) rotations, reading R4."""
    n = phi.shape[0]
    cp, sp = np.cos(phi), np.sin(phi)
    ct, st = np.cos(theta), np.sin(theta)
    D = np.zeros((n, 3, 3))
    D[:, 0, 0], D[:, 0, 1] = cp, sp
    D[:, 1, 0], D[:, 1, 1] = -sp, cp
    D[:, 2, 2] = 1.0
    C = np.zeros((n, 3, 3))
    C[:, 0, 0], C[:, 0, 2] = ct, -st
    C[:, 1, 1] = 1.0
    C[:, 2, 0], C[:, 2, 2] = st, ct
    B = np.broadcast_to(np.eye(3), (n, 3, 3))
    return B @ C @ D


def rotated_tensor(N_eff: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Eq. (nrot): N_rot = R^T N_eff R."""
    return np.transpose(R, (0, 2, 1)) @ N_eff @ R


def e_field(alpha: float) -> np.ndarray:
    """e = U(alpha) (1, 0, 0): the beam's electric field rotated about z."""
    return U_matrix(alpha) @ np.array([1.0, 0.0, 0.0])


def U_matrix(alpha: float) -> np.ndarray:
    c, s = math.cos(alpha), math.sin(alpha)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def polarization(M: np.ndarray, nt: np.ndarray, e: np.ndarray,
                 chunk: int = 1 << 18) -> np.ndarray:
    """Eq. (polarization): p = sum_j (N_rot^j N_rot^j - I) e / (4 pi).

    M  : [c][Nz][Ny][Nx][4] (v, s, phi, theta), any float type (read as f64)
    nt : [c][4] (delta_par, beta_par, delta_perp, beta_perp) at this energy
    e  : (3,) real
    Returns p as [3][Nz][Ny][Nx] complex128 (component-major, R11)."""
    c = M.shape[0]
    grid = M.shape[1:4]
    nvox = int(np.prod(grid))
    Mf = M.reshape(c, nvox, 4)
    p = np.zeros((nvox, 3), dtype=np.complex128)
    I3 = np.eye(3)
    for j in range(c):
        N = refractive_tensor(*[float(x) for x in nt[j]])
        for lo in range(0, nvox, chunk):
            hi = min(nvox, lo + chunk)
            blk = Mf[j, lo:hi].astype(np.float64)
            N_eff = effective_tensor(N, blk[:, 0], blk[:, 1])
            R = euler_R(blk[:, 2], blk[:, 3])
            N_rot = rotated_tensor(N_eff, R)
            A = N_rot @ N_rot - I3[None]
            p[lo:hi] += (A @ e) / (4.0 * math.pi)
    return np.ascontiguousarray(p.T).reshape((3,) + grid)


def rotate_back(p: np.ndarray, alpha: float) -> np.ndarray:
    """p <- U^T p (Sec. 3.3, Algorithm 1), applied to the components."""
    UT = U_matrix(alpha).T
    return np.einsum("ab,b...->a...", UT, p)


def fft3(p: np.ndarray) -> np.ndarray:
    """p~ = FFT(p) per component over (z, y, x); forward, unnormalised (R9)."""
    return np.fft.fftn(p, axes=(1, 2, 3))


def q_axis(n: int, voxel_nm: float) -> np.ndarray:
    """q values 2 pi m / (n Delta) in FFT order (m = 0..n/2-1, -n/2..-1)."""
    return 2.0 * math.pi * np.fft.fftfreq(n, d=voxel_nm)


def ewald(pt: np.ndarray, E_eV: float, voxel_nm: float) -> np.ndarray:
    """Eqs. (3Dscatter) and (Ewald): detector image in FFT order, [Ny][Nx].

    For every detector pixel (q_x, q_y): k_in = (0, 0, k); q_z from Eq.
    (Ewald) with |k_out| = k; zero when the root is imaginary (R10).
    k_out = k_in + q, r-hat = k_out / |k_out|.  X is interpolated linearly
    in q_z between the two nearest integer bins (R8):
        X = (1 - w) |Y(z0)|^2 + w |Y(z0 + 1)|^2,
        Y(b) = |k_out|^2 (I - r r) . p~(q_x, q_y, b).
    """
    _, Nz, Ny, Nx = pt.shape
    k = wavenumber(E_eV)
    qx = q_axis(Nx, voxel_nm)[None, :]
    qy = q_axis(Ny, voxel_nm)[:, None]
    dqz = 2.0 * math.pi / (Nz * voxel_nm)
    rad = k * k - qx * qx - qy * qy
    valid = rad >= 0.0
    qz = np.where(valid, -k + np.sqrt(np.where(valid, rad, 0.0)), 0.0)
    t = qz / dqz
    z0 = np.floor(t)
    w = t - z0
    b0 = np.mod(z0.astype(np.int64), Nz)
    b1 = np.mod(z0.astype(np.int64) + 1, Nz)
    kout = np.stack([np.broadcast_to(qx, qz.shape), np.broadcast_to(qy, qz.shape), k + qz])
    kmag = np.sqrt((kout ** 2).sum(axis=0))
    r = kout / kmag
    iy, ix = np.meshgrid(np.arange(Ny), np.arange(Nx), indexing="ij")
    X = np.zeros((Ny, Nx))
    for b, wt in ((b0, 1.0 - w), (b1, w)):
        v = pt[:, b, iy, ix]                       # (3, Ny, Nx) complex
        rv = (r * v).sum(axis=0)                   # r . p~
        Y = (kmag ** 2) * (v - r * rv)             # |k_out|^2 (I - r r) . p~
        X += wt * (np.abs(Y) ** 2).sum(axis=0)
    return np.where(valid, X, 0.0)


def dft_sparse(vals: np.ndarray, iz, iy, ix, shape, kz, ky, kx) -> np.ndarray:
    """The forward DFT (R9) by its definition, for a field that is zero
    except at the voxels (iz, iy, ix):
        p~(k) = sum_v p_v exp(-2 pi i (kz z_v / Nz + ky y_v / Ny + kx x_v / Nx)),
    at the frequency indices (kz[m], ky[m], kx[m]).  vals: [3][K] complex.
    Returns [3][P].  The integer products are reduced modulo N before the
    division, so the phases stay exact for large grids."""
    Nz, Ny, Nx = shape
    kz, ky, kx = (np.asarray(a, dtype=np.int64) for a in (kz, ky, kx))
    ph = (np.mod(np.outer(kz, iz), Nz) / Nz + np.mod(np.outer(ky, iy), Ny) / Ny
          + np.mod(np.outer(kx, ix), Nx) / Nx)
    return vals @ np.exp(-2j * math.pi * ph).T


def ewald_pixels(bins_fn, E_eV: float, voxel_nm: float, shape, iy, ix) -> np.ndarray:
    """Eqs. (3Dscatter) and (Ewald) at selected detector pixels (FFT-order
    indices iy, ix): the geometry and interpolation of ewald(), with p~ at
    the two q_z bins supplied by bins_fn(b, iy, ix) -> [3][P] complex."""
    Nz, Ny, Nx = shape
    iy, ix = np.asarray(iy), np.asarray(ix)
    k = wavenumber(E_eV)
    qx = q_axis(Nx, voxel_nm)[ix]
    qy = q_axis(Ny, voxel_nm)[iy]
    dqz = 2.0 * math.pi / (Nz * voxel_nm)
    rad = k * k - qx * qx - qy * qy
    valid = rad >= 0.0
    qz = np.where(valid, -k + np.sqrt(np.where(valid, rad, 0.0)), 0.0)
    t = qz / dqz
    z0 = np.floor(t)
    w = t - z0
    b0 = np.mod(z0.astype(np.int64), Nz)
    b1 = np.mod(z0.astype(np.int64) + 1, Nz)
    kout = np.stack([qx, qy, k + qz])
    kmag = np.sqrt((kout ** 2).sum(axis=0))
    r = kout / kmag
    X = np.zeros(iy.shape)
    for b, wt in ((b0, 1.0 - w), (b1, w)):
        v = bins_fn(b, iy, ix)                     # (3, P) complex
        rv = (r * v).sum(axis=0)
        Y = (kmag ** 2) * (v - r * rv)
        X += wt * (np.abs(Y) ** 2).sum(axis=0)
    return np.where(valid, X, 0.0)


def scatter_sparse_pixels(sparse, shape, nt, E_eV, voxel_nm, alpha, iy, ix,
                          uT_mode="literal") -> np.ndarray:
    """scatter_one_angle at selected pixels (FFT-order iy, ix) for a
    morphology that is vacuum (last component) except at sparse voxels
    (synth.sparse_voxels): p is the vacuum value p_vac everywhere else, so by
    linearity of the DFT p~(k) = DFT(p - p_vac)(k) + N p_vac [k = 0], and
    the first term is a sum over the sparse voxels (dft_sparse)."""
    iz_v, iy_v, ix_v, vals = sparse
    c = vals.shape[0]
    e = e_field(alpha)
    p = polarization(vals[:, None, None, :, :], nt, e)[:, 0, 0, :]    # (3, K)
    vac = np.zeros((c, 1, 1, 1, 4))
    vac[-1, ..., 0] = 1.0
    p_vac = polarization(vac, nt, e)[:, 0, 0, 0]                       # (3,)
    if uT_mode == "literal":
        p = rotate_back(p, alpha)
        p_vac = rotate_back(p_vac, alpha)
    dp = p - p_vac[:, None]
    N = int(np.prod(shape))

    def bins_fn(b, qy_i, qx_i):
        out = dft_sparse(dp, iz_v, iy_v, ix_v, shape, b, qy_i, qx_i)
        at0 = (np.asarray(b) == 0) & (np.asarray(qy_i) == 0) & (np.asarray(qx_i) == 0)
        return out + np.outer(p_vac * N, at0)

    return ewald_pixels(bins_fn, E_eV, voxel_nm, shape, iy, ix)


def fftshift2(img: np.ndarray) -> np.ndarray:
    """Detector image in fftshift order: q = 0 at index (Ny//2, Nx//2)."""
    return np.fft.fftshift(img, axes=(0, 1))


def rotate_image(img: np.ndarray, alpha: float) -> np.ndarray:
    """Rotated detector image (R6): out(Q) = img(U(alpha) Q), bilinear.

    img is in fftshift order.  Q is a physical q vector; with q_x spacing
    2 pi/(Nx Delta) and q_y spacing 2 pi/(Ny Delta) the map in pixel units
    is fx = cx + cos a (ix - cx) - sin a (Nx/Ny)(iy - cy),
       fy = cy + sin a (Ny/Nx)(ix - cx) + cos a (iy - cy),
    with cx = Nx//2, cy = Ny//2.  Corners outside the grid read zero."""
    Ny, Nx = img.shape
    cx, cy = Nx // 2, Ny // 2
    ca, sa = math.cos(alpha), math.sin(alpha)
    iy, ix = np.meshgrid(np.arange(Ny, dtype=np.float64), np.arange(Nx, dtype=np.float64),
                         indexing="ij")
    fx = cx + ca * (ix - cx) - sa * (Nx / Ny) * (iy - cy)
    fy = cy + sa * (Ny / Nx) * (ix - cx) + ca * (iy - cy)
    x0 = np.floor(fx)
    y0 = np.floor(fy)
    tx = fx - x0
    ty = fy - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    out = np.zeros_like(img)
    for dy, wy in ((0, 1.0 - ty), (1, ty)):
        for dx, wx in ((0, 1.0 - tx), (1, tx)):
            xx, yy = x0 + dx, y0 + dy
            ok = (xx >= 0) & (xx < Nx) & (yy >= 0) & (yy < Ny)
            val = np.where(ok, img[np.clip(yy, 0, Ny - 1), np.clip(xx, 0, Nx - 1)], 0.0)
            out += wy * wx * val
    return out


def rotate_sampled(pixel_fn, shape2, alpha: float, oy, ox) -> np.ndarray:
    """rotate_image evaluated only at the output pixels (oy, ox) (fftshift
    order): the same source positions and bilinear weights (R6), with the
    unrotated image read through pixel_fn(sy, sx) -> values at fftshift-order
    pixels (called once, on the in-grid corners)."""
    Ny, Nx = shape2
    cx, cy = Nx // 2, Ny // 2
    ca, sa = math.cos(alpha), math.sin(alpha)
    ix = np.asarray(ox, dtype=np.float64)
    iy = np.asarray(oy, dtype=np.float64)
    fx = cx + ca * (ix - cx) - sa * (Nx / Ny) * (iy - cy)
    fy = cy + sa * (Ny / Nx) * (ix - cx) + ca * (iy - cy)
    x0 = np.floor(fx)
    y0 = np.floor(fy)
    tx = fx - x0
    ty = fy - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    corners = []
    for dy, wy in ((0, 1.0 - ty), (1, ty)):
        for dx, wx in ((0, 1.0 - tx), (1, tx)):
            xx, yy = x0 + dx, y0 + dy
            ok = (xx >= 0) & (xx < Nx) & (yy >= 0) & (yy < Ny)
            corners.append((yy, xx, wy * wx, ok))
    sy = np.concatenate([c[0][c[3]] for c in corners])
    sx = np.concatenate([c[1][c[3]] for c in corners])
    vals = np.asarray(pixel_fn(sy, sx), dtype=np.float64) if sy.size else np.zeros(0)
    out = np.zeros(ix.shape)
    pos = 0
    for yy, xx, wt, ok in corners:
        n = int(ok.sum())
        contrib = np.zeros(ix.shape)
        contrib[ok] = vals[pos:pos + n]
        pos += n
        out += wt * contrib
    return out


def run_alg1_sparse_pixels(sparse, shape, constants_e, E_eV, voxel_nm, angles_deg, oy, ox,
                           rotation=True, uT_mode="literal") -> np.ndarray:
    """Algorithm 1's Ewald_Avg for one energy at the output pixels (oy, ox)
    (fftshift order) of a vacuum-plus-sparse morphology: for each angle the
    unrotated image is evaluated (scatter_sparse_pixels) at the corners the
    rotation reads (rotate_sampled), then averaged over the angles."""
    Nz, Ny, Nx = shape
    alphas = angle_list(*angles_deg, rotation=rotation)
    acc = np.zeros(np.asarray(ox).shape)
    for a in alphas:
        def pix(sy, sx, a=a):
            return scatter_sparse_pixels(sparse, shape, constants_e, E_eV, voxel_nm, a,
                                         np.mod(sy - Ny // 2, Ny), np.mod(sx - Nx // 2, Nx),
                                         uT_mode)
        if rotation:
            acc += rotate_sampled(pix, (Ny, Nx), a, oy, ox)
        else:
            acc += pix(np.asarray(oy), np.asarray(ox))
    return acc / len(alphas)


def angle_list(start_deg: float, inc_deg: float, end_deg: float,
               rotation: bool = True) -> np.ndarray:
    """E_Angle = [start, increment, end] in degrees -> radians (R7).
    With rotation disabled the single angle 0 is used (e = (1, 0, 0))."""
    if not rotation:
        return np.zeros(1)
    n = int(math.floor((end_deg - start_deg) / inc_deg + 1e-6)) + 1
    return np.deg2rad(start_deg + inc_deg * np.arange(n))


def scatter_one_angle(M, nt, E_eV, voxel_nm, alpha, uT_mode="literal"):
    """One pass of Algorithm 1's inner loop: image (fftshift order, not yet
    rotated) for one energy and one e-field angle."""
    e = e_field(alpha)
    p = polarization(M, nt, e)
    if uT_mode == "literal":
        p = rotate_back(p, alpha)
    pt = fft3(p)
    return fftshift2(ewald(pt, E_eV, voxel_nm))


def run_alg1(M, constants, energies, voxel_nm, angles_deg=(0.0, 1.0, 0.0),
             rotation=True, uT_mode="literal", energy_indices=None):
    """Algorithm 1: Ewald_Avg[i] for every energy (or the selected ones).

    M          : [c][Nz][Ny][Nx][4]
    constants  : [n_E][c][4]
    energies   : [n_E] eV
    angles_deg : (start, increment, end)
    Returns [n_sel][Ny][Nx] float64, fftshift order."""
    alphas = angle_list(*angles_deg, rotation=rotation)
    sel = range(len(energies)) if energy_indices is None else energy_indices
    Ny, Nx = M.shape[2], M.shape[3]
    out = np.zeros((len(sel), Ny, Nx))
    for o, i in enumerate(sel):
        acc = np.zeros((Ny, Nx))
        for a in alphas:
            img = scatter_one_angle(M, constants[i], energies[i], voxel_nm, a, uT_mode)
            acc += rotate_image(img, a) if rotation else img
        out[o] = acc / len(alphas)
    return out


# ------------------------------------------------------ Sec. 4.3 (Alg. 2, 3)
def nr_computation(M: np.ndarray, nt: np.ndarray, chunk: int = 1 << 18) -> np.ndarray:
    """Algorithm 3 (NrComputation): per voxel, loop over the components and
    accumulate N_t += (N_r^j N_r^j - I) / (4 pi), with N_r^j from Eqs. (ncorr)
    and (nrot).  Returns N_t as [Nz][Ny][Nx][3][3] complex128."""
    c = M.shape[0]
    grid = M.shape[1:4]
    nvox = int(np.prod(grid))
    Mf = M.reshape(c, nvox, 4)
    Nt = np.zeros((nvox, 3, 3), dtype=np.complex128)
    I3 = np.eye(3)
    for j in range(c):
        N = refractive_tensor(*[float(x) for x in nt[j]])
        for lo in range(0, nvox, chunk):
            hi = min(nvox, lo + chunk)
            blk = Mf[j, lo:hi].astype(np.float64)
            N_rot = rotated_tensor(effective_tensor(N, blk[:, 0], blk[:, 1]),
                                   euler_R(blk[:, 2], blk[:, 3]))
            Nt[lo:hi] += (N_rot @ N_rot - I3[None]) / (4.0 * math.pi)
    return Nt.reshape(grid + (3, 3))


def polarization_from_nt(Nt: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Algorithm 2: p(x) = N_t(x) . e_rot, returned as [3][Nz][Ny][Nx]."""
    return np.moveaxis(Nt @ e, -1, 0)


def run_alg2(M, constants, energies, voxel_nm, angles_deg=(0.0, 1.0, 0.0),
             rotation=True, uT_mode="literal", energy_indices=None):
    """Algorithm 2: N_t computed once per energy (Algorithm 3), then per
    e-field angle p = N_t . e, p <- U^T p, FFT, Ewald, rotation, average."""
    alphas = angle_list(*angles_deg, rotation=rotation)
    sel = range(len(energies)) if energy_indices is None else energy_indices
    Ny, Nx = M.shape[2], M.shape[3]
    out = np.zeros((len(sel), Ny, Nx))
    for o, i in enumerate(sel):
        Nt = nr_computation(M, constants[i])
        acc = np.zeros((Ny, Nx))
        for a in alphas:
            p = polarization_from_nt(Nt, e_field(a))
            if uT_mode == "literal":
                p = rotate_back(p, a)
            img = fftshift2(ewald(fft3(p), energies[i], voxel_nm))
            acc += rotate_image(img, a) if rotation else img
        out[o] = acc / len(alphas)
    return out


# ------------------------------------- linearity restatement of Algorithm 2
def run_linear(M, constants, energies, voxel_nm, angles_deg=(0.0, 1.0, 0.0),
               rotation=True, uT_mode="literal", energy_indices=None):
    """Algorithm 2 rewritten with the linearity of p in e and of the FFT:
    e(alpha) = cos(alpha) x + sin(alpha) y, so
        p~(alpha) = FFT(N_t x) cos(alpha) + FFT(N_t y) sin(alpha),
    then U^T, Eqs. (3Dscatter), (Ewald), rotation and average as before.
    The two FFT'd columns of N_t are formed once per energy."""
    alphas = angle_list(*angles_deg, rotation=rotation)
    sel = range(len(energies)) if energy_indices is None else energy_indices
    Ny, Nx = M.shape[2], M.shape[3]
    out = np.zeros((len(sel), Ny, Nx))
    for o, i in enumerate(sel):
        Nt = nr_computation(M, constants[i])
        Fx = fft3(np.moveaxis(Nt[..., :, 0], -1, 0))   # FFT of N_t x-hat
        Fy = fft3(np.moveaxis(Nt[..., :, 1], -1, 0))   # FFT of N_t y-hat
        acc = np.zeros((Ny, Nx))
        for a in alphas:
            pt = math.cos(a) * Fx + math.sin(a) * Fy
            if uT_mode == "literal":
                pt = rotate_back(pt, a)
            img = fftshift2(ewald(pt, energies[i], voxel_nm))
            acc += rotate_image(img, a) if rotation else img
        out[o] = acc / len(alphas)
    return out
