"""Seeded synthetic inputs for the P-RSoXS forward model.

This module only draws numbers: morphologies (per-voxel v_frac, s, phi, theta
for each component, the four features of Sec. 3.1) and optical-constant
tables (delta, beta along and across the extraordinary axis, per energy and
component, Sec. 3.2).  It holds none of the scattering arithmetic, so both the
CUDA path and the CPU oracle can be fed from it.

Layouts
-------
morphology : float array [c][Nz][Ny][Nx][4], last axis (v_frac, s, phi, theta),
             component-major as in the memory layout of Sec. 4.1 (Fig. 3),
             x fastest within a component.
constants  : float64 array [n_E][c][4], last axis
             (delta_par, beta_par, delta_perp, beta_perp).

The paper's optical constants (polyethylene, PEOlig, polystyrene, gold) and
its HDF5 morphologies are not available, so every input here is synthetic:
smooth resonant spectra near the carbon K edge and random multi-component
partitions of the box.
"""
from __future__ import annotations

import numpy as np

CARBON_EDGE_EV = 285.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def energies_uniform(n: int, lo: float = 270.0, hi: float = 320.0) -> np.ndarray:
    """n photon energies (eV) evenly spaced on [lo, hi]."""
    if n == 1:
        return np.array([0.5 * (lo + hi)])
    return np.linspace(lo, hi, n)


def _lorentz(E, E0, gamma):
    return (0.5 * gamma) ** 2 / ((E - E0) ** 2 + (0.5 * gamma) ** 2)


def optical_constants(energies, n_components: int, seed: int = 0,
                      vacuum_last: bool = True) -> np.ndarray:
    """Resonant delta(E), beta(E) pairs per component, [n_E][c][4] float64.

    Each non-vacuum component gets a background delta0 ~ U[1e-4, 1e-3] and
    beta0 ~ U[1e-5, 1e-4] with a small linear slope, plus a Lorentzian
    resonance near 285 eV.  The parallel and perpendicular responses differ by
    an amplitude factor U[0.5, 1.5], which makes the component birefringent.
    The last component is vacuum (all four constants zero) when vacuum_last.
    """
    E = np.asarray(energies, dtype=np.float64)
    g = rng(seed)
    out = np.zeros((E.size, n_components, 4))
    n_mat = n_components - 1 if (vacuum_last and n_components > 1) else n_components
    for j in range(n_mat):
        d0, b0 = g.uniform(1e-4, 1e-3), g.uniform(1e-5, 1e-4)
        slope = g.uniform(-2e-7, 2e-7)
        E0 = CARBON_EDGE_EV + g.uniform(-3.0, 3.0)
        gam = g.uniform(1.0, 4.0)
        amp_b = g.uniform(1e-3, 5e-3)
        amp_d = g.uniform(5e-4, 2e-3)
        aniso = g.uniform(0.5, 1.5, size=2)
        L = _lorentz(E, E0, gam)
        # dispersive partner of the Lorentzian: odd in (E - E0)
        D = (E - E0) * (0.5 * gam) / ((E - E0) ** 2 + (0.5 * gam) ** 2)
        delta_base = d0 + slope * (E - CARBON_EDGE_EV)
        out[:, j, 0] = delta_base + aniso[0] * amp_d * D
        out[:, j, 1] = b0 + aniso[0] * amp_b * L
        out[:, j, 2] = delta_base + aniso[1] * amp_d * D
        out[:, j, 3] = b0 + aniso[1] * amp_b * L
    return out


def morphology_random(shape, n_components: int, seed: int = 0,
                      binary: bool = False, dtype=np.float32) -> np.ndarray:
    """Random c-component morphology on a (Nz, Ny, Nx) grid.

    Volume fractions: smoothed noise fields turned into a partition of unity
    (fractional), or the arg-max of those fields (binary, one component per
    voxel).  s ~ U[0, 1] (or {0, 1} when binary), phi ~ U[0, 2 pi),
    theta ~ U[0, pi].
    """
    Nz, Ny, Nx = shape
    c = n_components
    g = rng(seed)
    M = np.empty((c, Nz, Ny, Nx, 4), dtype=dtype)
    # Smooth noise by box-averaging white noise over a few voxels per axis
    # (periodic), which gives the partition some domain structure.
    fields = g.random((c, Nz, Ny, Nx), dtype=np.float32)
    for ax, n in ((1, Nz), (2, Ny), (3, Nx)):
        w = min(3, n)
        acc = np.zeros_like(fields)
        for sh in range(w):
            acc += np.roll(fields, sh - w // 2, axis=ax)
        fields = acc / w
    if binary:
        win = np.argmax(fields, axis=0)
        for j in range(c):
            M[j, ..., 0] = (win == j)
    else:
        f = fields ** 4
        M[..., 0] = (f / f.sum(axis=0, keepdims=True))
    if binary:
        M[..., 1] = g.integers(0, 2, size=(c, Nz, Ny, Nx))
    else:
        M[..., 1] = g.random((c, Nz, Ny, Nx), dtype=np.float32)
    M[..., 2] = g.uniform(0.0, 2.0 * np.pi, size=(c, Nz, Ny, Nx))
    M[..., 3] = g.uniform(0.0, np.pi, size=(c, Nz, Ny, Nx))
    return M


def _empty(shape, c, dtype):
    Nz, Ny, Nx = shape
    return np.zeros((c, Nz, Ny, Nx, 4), dtype=dtype)


def morphology_sphere(shape, radius_vox: float, dtype=np.float64) -> np.ndarray:
    """Two components: an isotropic sphere (component 0) in vacuum
    (component 1), centred in the box; binary volume fractions."""
    Nz, Ny, Nx = shape
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    cz, cy, cx = (Nz - 1) / 2, (Ny - 1) / 2, (Nx - 1) / 2
    inside = ((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) <= radius_vox ** 2
    M = _empty(shape, 2, dtype)
    M[0, ..., 0] = inside
    M[1, ..., 0] = ~inside
    return M


def morphology_disk(shape, radius_vox: float, dtype=np.float64) -> np.ndarray:
    """Two components: an isotropic cylinder along z (a disk in every
    z-slice) in vacuum; binary volume fractions."""
    Nz, Ny, Nx = shape
    y, x = np.meshgrid(np.arange(Ny), np.arange(Nx), indexing="ij")
    cy, cx = (Ny - 1) / 2, (Nx - 1) / 2
    inside = ((x - cx) ** 2 + (y - cy) ** 2) <= radius_vox ** 2
    M = _empty(shape, 2, dtype)
    M[0, ..., 0] = inside[None]
    M[1, ..., 0] = ~inside[None]
    return M


def morphology_hex_lattice(shape, spacing_vox: float, radius_vox: float,
                           dtype=np.float64) -> np.ndarray:
    """Two components: isotropic disks on a 2-D hexagonal lattice (nearest
    neighbour distance spacing_vox), cylinders parallel to the beam, in vacuum."""
    Nz, Ny, Nx = shape
    y, x = np.meshgrid(np.arange(Ny, dtype=np.float64), np.arange(Nx, dtype=np.float64),
                       indexing="ij")
    a = spacing_vox
    b = a * np.sqrt(3.0)
    inside = np.zeros((Ny, Nx), dtype=bool)
    for base in ((0.0, 0.0), (0.5 * a, 0.5 * b)):
        for iy in range(-1, int(Ny / b) + 2):
            for ix in range(-1, int(Nx / a) + 2):
                px, py = base[0] + ix * a, base[1] + iy * b
                if -radius_vox - 1 <= px <= Nx + radius_vox and -radius_vox - 1 <= py <= Ny + radius_vox:
                    inside |= (x - px) ** 2 + (y - py) ** 2 <= radius_vox ** 2
    M = _empty(shape, 2, dtype)
    M[0, ..., 0] = inside[None]
    M[1, ..., 0] = ~inside[None]
    return M


def morphology_grating(shape, period_vox: int, width_vox: int, axis: str = "x",
                       dtype=np.float64) -> np.ndarray:
    """Two components: isotropic lines of width width_vox repeating every
    period_vox voxels along `axis`, uniform along the other axes."""
    Nz, Ny, Nx = shape
    M = _empty(shape, 2, dtype)
    if axis == "x":
        line = (np.arange(Nx) % period_vox) < width_vox
        M[0, ..., 0] = line[None, None, :]
    else:
        line = (np.arange(Ny) % period_vox) < width_vox
        M[0, ..., 0] = line[None, :, None]
    M[1, ..., 0] = 1.0 - M[0, ..., 0]
    return M


def morphology_random_torch(shape, n_components: int, seed: int = 0, device="cuda",
                            dtype=None):
    """Device-side counterpart of morphology_random for large grids (the
    benchmark's 10-GB morphologies): same recipe (smoothed-noise partition
    of unity for v, s ~ U[0,1], phi ~ U[0, 2 pi), theta ~ U[0, pi]), drawn
    with torch's seeded generator on `device`; not bitwise equal to the
    numpy version.  Returns a contiguous [c][Nz][Ny][Nx][4] tensor."""
    import torch

    dtype = dtype or torch.float32
    Nz, Ny, Nx = shape
    c = n_components
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    M = torch.empty((c, Nz, Ny, Nx, 4), device=device, dtype=dtype)
    fields = torch.rand((c, Nz, Ny, Nx), generator=g, device=device)
    for ax, n in ((1, Nz), (2, Ny), (3, Nx)):
        w = min(3, n)
        acc = torch.zeros_like(fields)
        for sh in range(w):
            acc += torch.roll(fields, sh - w // 2, dims=ax)
        fields = acc / w
        del acc
    fields = fields ** 4
    fields /= fields.sum(dim=0, keepdim=True)
    M[..., 0] = fields
    del fields
    M[..., 1] = torch.rand((c, Nz, Ny, Nx), generator=g, device=device)
    M[..., 2] = torch.rand((c, Nz, Ny, Nx), generator=g, device=device) * (2.0 * np.pi)
    M[..., 3] = torch.rand((c, Nz, Ny, Nx), generator=g, device=device) * np.pi
    return M


def sparse_voxels(shape, n_components: int, n_voxels: int, seed: int = 0):
    """A morphology that is vacuum (the last component, v = 1) everywhere
    except at about n_voxels distinct random voxels, which hold a random mix
    of all components (v a random partition of unity, s ~ U[0,1],
    phi ~ U[0, 2 pi), theta ~ U[0, pi]).  Returns (iz, iy, ix, vals) with
    vals [c][K][4] float64; dense forms: morphology_sparse(_torch)."""
    g = rng(seed)
    Nz, Ny, Nx = shape
    flat = np.unique(g.integers(0, Nz * Ny * Nx, size=n_voxels))
    iz, rem = np.divmod(flat, Ny * Nx)
    iy, ix = np.divmod(rem, Nx)
    K, c = flat.size, n_components
    v = g.random((c, K)) ** 2
    v /= v.sum(axis=0, keepdims=True)
    vals = np.empty((c, K, 4))
    vals[..., 0] = v
    vals[..., 1] = g.random((c, K))
    vals[..., 2] = g.random((c, K)) * (2.0 * np.pi)
    vals[..., 3] = g.random((c, K)) * np.pi
    return iz, iy, ix, vals


def morphology_sparse(shape, n_components: int, sparse, dtype=np.float64) -> np.ndarray:
    """Dense [c][Nz][Ny][Nx][4] form of sparse_voxels' output."""
    iz, iy, ix, vals = sparse
    M = np.zeros((n_components,) + tuple(shape) + (4,), dtype=dtype)
    M[-1, ..., 0] = 1.0
    M[:, iz, iy, ix, :] = vals
    return M


def morphology_sparse_torch(shape, n_components: int, sparse, device="cuda", dtype=None):
    """Device-side dense form of sparse_voxels' output (for full-size grids)."""
    import torch

    dtype = dtype or torch.float32
    iz, iy, ix, vals = sparse
    M = torch.zeros((n_components,) + tuple(shape) + (4,), device=device, dtype=dtype)
    M[-1, ..., 0] = 1.0
    idx = [torch.as_tensor(a, device=device) for a in (iz, iy, ix)]
    M[:, idx[0], idx[1], idx[2], :] = torch.as_tensor(vals, device=device, dtype=dtype)
    return M
