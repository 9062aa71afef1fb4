"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no step of the lattice Boltzmann method: it only draws
random numbers and shapes them into input fields and parameter sets.  The
paper (arXiv:1308.2071) measures on no dataset; every workload here is
synthetic and reproducible from its seed.

- ``porosity_field``: a heterogeneous porosity field whose permeability is
  log-normal with a Gaussian covariance (correlation length in cells).  The
  permeability is mapped to porosity through the monotone shape of Ergun's
  relation, K proportional to phi^3 / (1 - phi)^2 (Section 2, Eq. 5), anchored so
  that the mean porosity gives the mean permeability, then clipped.  This is
  how the input is constructed; both the oracle and the CUDA library compute
  K(phi) and F_phi(phi) from the porosity on their own.
- ``perturbed_porosity``: a smooth seeded perturbation of a uniform porosity.
- ``cavity_sweep``: the parameter draws of a batched sweep of cavities.
"""
from __future__ import annotations

import numpy as np


def gaussian_random_field(ny: int, nx: int, corr_len: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field with covariance
    exp(-r^2 / (2 corr_len^2)), made by filtering white noise in Fourier space
    (FP64, periodic)."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k2 = (2.0 * np.pi) ** 2 * (kx * kx + ky * ky)
    # spectral density of a Gaussian covariance is Gaussian; filter = its square root
    filt = np.exp(-0.25 * k2 * corr_len * corr_len)
    y = np.fft.irfft2(np.fft.rfft2(noise) * filt, s=(ny, nx))
    y -= y.mean()
    sd = y.std()
    return y / sd if sd > 0 else y


def _porosity_from_ratio(ratio: np.ndarray) -> np.ndarray:
    """Solves phi^3 / (1 - phi)^2 = ratio for phi in (0, 1) (FP64).  The left
    side in log form, g(phi) = 3 ln(phi) - 2 ln(1 - phi), is increasing, so a
    fine table of g inverted by linear interpolation gives a start within
    1e-11, and two Newton steps (g' = 3/phi + 2/(1 - phi)) reach full FP64."""
    grid = np.linspace(1e-7, 1.0 - 1e-7, 1 << 20)
    g_grid = 3.0 * np.log(grid) - 2.0 * np.log1p(-grid)
    target = np.log(ratio)
    phi = np.interp(target, g_grid, grid)
    for _ in range(2):
        g = 3.0 * np.log(phi) - 2.0 * np.log1p(-phi) - target
        phi = np.clip(phi - g / (3.0 / phi + 2.0 / (1.0 - phi)), 1e-12, 1.0 - 1e-12)
    return phi


def porosity_field(ny: int, nx: int, phi_bar: float = 0.6, corr_len: float = 32.0,
                   sigma_lnK: float = 1.0, clip=(0.3, 0.9), seed: int = 1308) -> np.ndarray:
    """Porosity field with log-normal permeability (ln K = ln K_bar + sigma_lnK * Y),
    Y a Gaussian random field of the given correlation length; returns FP64 (ny, nx)."""
    y = gaussian_random_field(ny, nx, corr_len, seed)
    ratio_bar = phi_bar ** 3 / (1.0 - phi_bar) ** 2
    phi = _porosity_from_ratio(ratio_bar * np.exp(sigma_lnK * y))
    return np.clip(phi, clip[0], clip[1])


def perturbed_porosity(ny: int, nx: int, phi_bar: float = 0.6, amplitude: float = 0.05,
                       corr_len: float = 8.0, seed: int = 2000) -> np.ndarray:
    """phi_bar plus a smooth seeded perturbation of the given amplitude (FP64)."""
    y = gaussian_random_field(ny, nx, corr_len, seed)
    return phi_bar + amplitude * np.tanh(y)


def random_state(ny: int, nx: int, seed: int, amp_f: float = 1e-3, amp_g: float = 1e-2):
    """Small seeded perturbations (9, ny, nx) and (5, ny, nx) to add to a rest state."""
    rng = np.random.default_rng(seed)
    return (amp_f * rng.standard_normal((9, ny, nx)), amp_g * rng.standard_normal((5, ny, nx)))


def cavity_sweep(n: int = 256, seed: int = 2071, size_range=(64, 512), Ra_range=(1e3, 1e6),
                 Da_range=(1e-4, 1e-1), phi_range=(0.3, 0.9)):
    """Parameter draws of a batched sweep: square cavities of uneven size,
    log-uniform Ra and Da, uniform porosity.  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(size_range[0], size_range[1] + 1, size=n)
    Ra = 10.0 ** rng.uniform(np.log10(Ra_range[0]), np.log10(Ra_range[1]), size=n)
    Da = 10.0 ** rng.uniform(np.log10(Da_range[0]), np.log10(Da_range[1]), size=n)
    phi = rng.uniform(phi_range[0], phi_range[1], size=n)
    return [dict(nx=int(s), ny=int(s), Ra=float(r), Da=float(d), phi=float(p))
            for s, r, d, p in zip(sizes, Ra, Da, phi)]
