"""The seeded input generators do what their recipe states (no GPU): the
Gaussian random field's moments and covariance, the inversion of Ergun's
porosity-permeability shape (Eq. 5), the clipped log-normal porosity field,
and the reproducible parameter draws of the batched sweep."""
import numpy as np
import pytest

from paper_1308_2071_gb300 import inputs


def test_gaussian_random_field_has_unit_variance_and_gaussian_covariance():
    n, corr = 512, 6.0
    y = inputs.gaussian_random_field(n, n, corr, seed=5)
    assert abs(y.mean()) < 1e-12 and abs(y.std() - 1.0) < 1e-12
    # periodic autocovariance from the power spectrum, against exp(-r^2 / (2 l^2))
    ac = np.fft.irfft2(np.abs(np.fft.rfft2(y)) ** 2, s=y.shape) / y.size
    for r in (0, 2, 4, 6, 9, 12):
        want = np.exp(-r * r / (2 * corr * corr))
        got = 0.5 * (ac[0, r] + ac[r, 0])
        assert abs(got - want) < 0.06, (r, got, want)
    assert np.array_equal(y, inputs.gaussian_random_field(n, n, corr, seed=5))  # seeded


def test_ergun_shape_is_inverted_to_full_precision():
    phi = np.linspace(0.05, 0.98, 4001)
    ratio = phi ** 3 / (1 - phi) ** 2
    back = inputs._porosity_from_ratio(ratio)
    assert np.abs(back - phi).max() < 1e-14
    assert np.all(np.diff(back) > 0)


def test_porosity_field_is_log_normal_in_permeability_and_clipped():
    ny, nx, phi_bar, corr = 96, 128, 0.6, 8.0
    phi = inputs.porosity_field(ny, nx, phi_bar=phi_bar, corr_len=corr, sigma_lnK=1.0, seed=1308)
    assert phi.shape == (ny, nx) and phi.min() >= 0.3 and phi.max() <= 0.9
    y = inputs.gaussian_random_field(ny, nx, corr, 1308)
    inside = (phi > 0.3) & (phi < 0.9)
    assert inside.mean() > 0.8
    # K proportional to phi^3 / (1 - phi)^2 (Eq. 5): ln K - ln K_bar = Y where not clipped
    lnK = 3 * np.log(phi) - 2 * np.log1p(-phi) - (3 * np.log(phi_bar) - 2 * np.log1p(-phi_bar))
    assert np.abs(lnK[inside] - y[inside]).max() < 1e-12
    # clipped cells are the ones whose unclipped porosity left the range
    assert np.all(y[phi == 0.9] > 0) and np.all(y[phi == 0.3] < 0)


@pytest.mark.parametrize("amplitude", [0.05, 0.1])
def test_perturbed_porosity_stays_within_its_amplitude(amplitude):
    phi = inputs.perturbed_porosity(40, 48, phi_bar=0.6, amplitude=amplitude, corr_len=6.0, seed=5)
    assert np.all(np.abs(phi - 0.6) < amplitude) and phi.std() > 0.2 * amplitude


def test_cavity_sweep_draws_are_reproducible_and_in_range():
    a = inputs.cavity_sweep(256, seed=2071)
    assert a == inputs.cavity_sweep(256, seed=2071) and a != inputs.cavity_sweep(256, seed=2072)
    n = np.array([c["nx"] for c in a])
    assert np.all(n == np.array([c["ny"] for c in a])) and n.min() >= 64 and n.max() <= 512
    Ra = np.array([c["Ra"] for c in a])
    Da = np.array([c["Da"] for c in a])
    phi = np.array([c["phi"] for c in a])
    assert Ra.min() >= 1e3 and Ra.max() <= 1e6 and Da.min() >= 1e-4 and Da.max() <= 1e-1
    assert phi.min() >= 0.3 and phi.max() <= 0.9
    # log-uniform: log10 Ra spread over the three decades
    assert np.histogram(np.log10(Ra), bins=3, range=(3, 6))[0].min() > 50
