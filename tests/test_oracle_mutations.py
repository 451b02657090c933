"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's source (a transposed
operand, a dropped term, a wrong sign or index, a changed reading) and runs
the pin tests against the mutated copy: at least one pin must fail.  The
real oracle module is never modified."""
import inspect
import os
import types

import pytest

from oracle import cyrsoxs_oracle
import tests.test_oracle_pins as pins
import tests.test_grating_trapezoid as grating

SRC = inspect.getsource(cyrsoxs_oracle)

MUTANTS = {
    "R transposed": ("    return B @ C @ D", "    return np.transpose(B @ C @ D, (0, 2, 1))"),
    "sign of sin(theta) in C": ("C[:, 0, 0], C[:, 0, 2] = ct, -st", "C[:, 0, 0], C[:, 0, 2] = ct, st"),
    "unaligned part dropped": ("(1.0 - s)[:, None, None] * iso[None]", "(0.0 * s)[:, None, None] * iso[None]"),
    "trace not divided by 3": ("iso = np.trace(N) / 3.0 * np.eye(3)", "iso = np.trace(N) * np.eye(3)"),
    "R N R^T instead of R^T N R": ("return np.transpose(R, (0, 2, 1)) @ N_eff @ R",
                                   "return R @ N_eff @ np.transpose(R, (0, 2, 1))"),
    "identity not subtracted": ("A = N_rot @ N_rot - I3[None]", "A = N_rot @ N_rot"),
    "U instead of U^T": ("UT = U_matrix(alpha).T", "UT = U_matrix(alpha)"),
    "inverse FFT sign": ("return np.fft.fftn(p, axes=(1, 2, 3))",
                         "return np.fft.ifftn(p, axes=(1, 2, 3)) * np.prod(p.shape[1:])"),
    "sign of q_z": ("qz = np.where(valid, -k + np.sqrt", "qz = np.where(valid, k - np.sqrt"),
    "interpolation weights swapped": ("for b, wt in ((b0, 1.0 - w), (b1, w)):",
                                      "for b, wt in ((b0, w), (b1, 1.0 - w)):"),
    "projection sign": ("Y = (kmag ** 2) * (v - r * rv)", "Y = (kmag ** 2) * (v + r * rv)"),
    "upper bin off by one": ("b1 = np.mod(z0.astype(np.int64) + 1, Nz)",
                             "b1 = np.mod(z0.astype(np.int64) + 2, Nz)"),
    "rotation direction": ("fx = cx + ca * (ix - cx) - sa * (Nx / Ny) * (iy - cy)",
                           "fx = cx + ca * (ix - cx) + sa * (Nx / Ny) * (iy - cy)"),
    "bilinear weight": ("out += wy * wx * val", "out += wx * wx * val"),
    "angle list excludes end": ("n = int(math.floor((end_deg - start_deg) / inc_deg + 1e-6)) + 1",
                                "n = int(math.floor((end_deg - start_deg) / inc_deg + 1e-6))"),
    "sign of delta": ("n_par = 1.0 - delta_par + 1j * beta_par",
                      "n_par = 1.0 + delta_par + 1j * beta_par"),
    "extraordinary axis on x": ("np.diag(np.array([n_perp, n_perp, n_par], dtype=np.complex128))",
                                "np.diag(np.array([n_par, n_perp, n_perp], dtype=np.complex128))"),
    "wavenumber without 2 pi": ("return 2.0 * math.pi / wavelength_nm(E_eV)",
                                "return math.pi / wavelength_nm(E_eV)"),
    "average not divided": ("out[o] = acc / len(alphas)", "out[o] = acc"),  # Algorithm 1's
    "image not fftshifted": ("return np.fft.fftshift(img, axes=(0, 1))", "return img"),
    "sampled rotation reads corners in the wrong order": (
        "contrib[ok] = vals[pos:pos + n]", "contrib[ok] = vals[pos:pos + n][::-1]"),
    "sampled average not divided": ("    return acc / len(alphas)", "    return acc"),
    "sampled pixels not shifted back to FFT order": (
        "np.mod(sy - Ny // 2, Ny), np.mod(sx - Nx // 2, Nx)", "sy, sx"),
}


def _pin_functions():
    fns = []
    for mod in (pins, grating):
        for name, fn in sorted(vars(mod).items()):
            if name.startswith("test_") and callable(fn):
                sig = inspect.signature(fn)
                if not sig.parameters and not getattr(fn, "pytestmark", None):
                    fns.append(fn)
    return fns


def _mutant_module(old, new):
    assert SRC.count(old) >= 1, f"mutation site not found: {old!r}"
    src = SRC.replace(old, new, 1)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = os.path.abspath(cyrsoxs_oracle.__file__)
    exec(compile(src, "oracle_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    old, new = MUTANTS[name]
    mutant = _mutant_module(old, new)
    monkeypatch.setattr(pins, "O", mutant)
    monkeypatch.setattr(grating, "O", mutant)
    caught = []
    for fn in _pin_functions():
        try:
            fn()
        except (AssertionError, ValueError, ZeroDivisionError, IndexError, FloatingPointError):
            caught.append(fn.__name__)
            break
    assert caught, f"no pin fails with the mistake '{name}'"


def test_unmutated_oracle_passes_every_pin():
    for fn in _pin_functions():
        fn()
