"""Pins of the oracle's binned profiles (Table profile; reading R19: the average of the profile
over the grid bin centred on each grid point) against SciPy's independent special functions
and adaptive quadrature, the telescoping of bin masses into exact areas, and the limits to
the sampled profiles (fine bins) and between the profile kinds."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle

LN2 = math.log(2.0)


def _sigma(alpha):
    return alpha / math.sqrt(2 * LN2)


def test_binned_gauss_is_erf_difference():
    a, dnu = 0.037, 0.01
    x = np.linspace(-0.3, 0.3, 121)
    f = oracle.profile_binned("gauss_hwhm", x, dnu, a)
    c = math.sqrt(LN2) / a
    ref = 0.5 * (special.erf((x + dnu / 2) * c) - special.erf((x - dnu / 2) * c)) / dnu
    big = ref * dnu > 1e-6          # the plain erf difference cancels below that
    np.testing.assert_allclose(f[big], ref[big], rtol=1e-9, atol=0)
    # far tail (both edges on one side): erfc keeps full relative accuracy
    xt = np.array([0.25, 0.3, -0.3])
    ft = oracle.profile_binned("gauss_hwhm", xt, dnu, a)
    reft = np.array([0.5 * (special.erfc((abs(v) - dnu / 2) * c) - special.erfc((abs(v) + dnu / 2) * c)) / dnu
                     for v in xt])
    np.testing.assert_allclose(ft, reft, rtol=1e-12)


def test_binned_lorentz_matches_quadrature_and_arctangent():
    g, dnu = 0.02, 0.1
    x = np.concatenate([np.linspace(-2, 2, 81), [0.0, 0.05, -0.05, 30.0]])
    f = oracle.profile_binned("lorentz", x, dnu, 0.0, g)
    for xi, fi in zip(x, f):
        q, _ = integrate.quad(lambda u: g / (math.pi * (u * u + g * g)), xi - dnu / 2, xi + dnu / 2,
                              epsabs=0, epsrel=1e-13, limit=200)
        assert fi == pytest.approx(q / dnu, rel=1e-10)


@pytest.mark.parametrize("a,g,dnu", [(0.013, 0.002, 0.1), (0.05, 0.05, 0.01), (0.01, 0.3, 0.05),
                                     (0.2, 1e-4, 0.01)])
def test_binned_voigt_matches_scipy_quadrature(a, g, dnu):
    s = _sigma(a)
    x = np.array([0.0, 0.5 * dnu, 0.7 * dnu, 3 * dnu, -11.3 * dnu, 40 * dnu, 2.0])
    f = oracle.profile_binned("voigt", x, dnu, a, g)
    for xi, fi in zip(x, f):
        lo, hi = xi - dnu / 2, xi + dnu / 2
        pts = [0.0] if lo < 0 < hi else None
        q, _ = integrate.quad(lambda u: special.voigt_profile(u, s, g), lo, hi, points=pts,
                              epsabs=0, epsrel=1e-12, limit=400)
        assert fi == pytest.approx(q / dnu, rel=1e-9), (xi, fi, q / dnu)


@pytest.mark.parametrize("kind", ["gauss_hwhm", "lorentz", "voigt"])
def test_bin_masses_telescope_to_the_exact_area(kind):
    # sum over consecutive bins of mass = integral over their union (coarse, undersampled bins
    # included: this is what makes integral sigma = sum I hold on any grid, R14)
    a, g, dnu = 0.013, 0.004, 0.1
    x = np.arange(-250, 251) * dnu + 0.0371        # line centre off the grid
    total = oracle.profile_binned(kind, x, dnu, a, g).sum() * dnu
    lo, hi = x[0] - dnu / 2, x[-1] + dnu / 2
    if kind == "gauss_hwhm":
        c = math.sqrt(LN2) / a
        ref = 0.5 * (special.erf(hi * c) - special.erf(lo * c))
    elif kind == "lorentz":
        ref = (math.atan(hi / g) - math.atan(lo / g)) / math.pi
    else:
        s = _sigma(a)
        ref = sum(integrate.quad(lambda u: special.voigt_profile(u, s, g), p, q, epsabs=0, epsrel=1e-13,
                                 limit=400)[0] for p, q in ((lo, -0.5), (-0.5, 0.0), (0.0, 0.5), (0.5, hi)))
    assert total == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("kind", ["gauss_hwhm", "lorentz", "voigt"])
def test_fine_bins_approach_the_sampled_profile(kind):
    # bin average = f(x) + dnu^2 f''(x) / 24 + O(dnu^4)
    a, g = 0.05, 0.03
    x = np.array([0.01, 0.04, 0.09, 0.2])
    f0 = oracle.profile(kind, x, a, g)
    for dnu in (1e-3, 5e-4):
        fb = oracle.profile_binned(kind, x, dnu, a, g)
        h = 1e-3
        f2 = (oracle.profile(kind, x + h, a, g) - 2 * f0 + oracle.profile(kind, x - h, a, g)) / h ** 2
        np.testing.assert_allclose(fb, f0 + dnu ** 2 * f2 / 24, rtol=1e-6)


def test_binned_voigt_limits():
    x = np.linspace(-0.4, 0.4, 33) + 0.003
    dnu = 0.02
    # gamma -> 0: the Gaussian, up to the Lorentz wings gamma / (pi x^2) ~ 1e-8 left by gamma = 1e-9
    np.testing.assert_allclose(oracle.profile_binned("voigt", x, dnu, 0.05, 1e-9),
                               oracle.profile_binned("gauss_hwhm", x, dnu, 0.05), rtol=1e-6, atol=3e-8)
    np.testing.assert_allclose(oracle.profile_binned("voigt", x, dnu, 1e-7, 0.03),
                               oracle.profile_binned("lorentz", x, dnu, 0.0, 0.03), rtol=1e-6)


def test_binned_cross_section_integral_equals_intensity_on_a_coarse_grid():
    # the doppler_1e5 configuration's 0.1 cm^-1 grid undersamples its ~0.013 cm^-1 Doppler widths;
    # binned profiles conserve sum(sigma) dnu = sum(I) for lines whose window holds the profile
    rng = np.random.default_rng(2)
    n = 40
    nu = rng.uniform(100.0, 900.0, n)
    I = 10.0 ** rng.uniform(-22, -19, n)
    alpha = nu * 3e-6
    gamma = np.full(n, 0.004)
    keep = np.ones(n, np.uint8)
    dnu, n_grid, cut = 0.1, 10001, 25.0
    ilo = np.ceil((nu - cut) / dnu).astype(np.int64)
    ihi = np.floor((nu + cut) / dnu).astype(np.int64)
    for kind in ("binned_gauss_doppler", "binned_voigt"):
        sig = oracle.cross_section(kind, nu, I, alpha, gamma, keep, ilo, ihi, 0.0, dnu, n_grid)
        expect = I.sum() if kind == "binned_gauss_doppler" else None
        if expect is None:   # Voigt: subtract the Lorentz wings beyond +-cut (closed form bound)
            tail = np.sum(I * (1 - 2 * np.arctan((cut + dnu / 2) / gamma) / np.pi))
            assert abs(sig.sum() * dnu - I.sum()) <= 1.05 * tail + 1e-12 * I.sum()
        else:
            assert sig.sum() * dnu == pytest.approx(expect, rel=1e-12)
