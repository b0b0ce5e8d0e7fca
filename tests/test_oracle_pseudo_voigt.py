"""Pins of the oracle's pseudo-Voigt profiles (Table profile; reading R20 in oracle/oracle.c).

Each pseudo-Voigt is a Lorentzian and a Gaussian of one common full width G, mixed with
weights w_L, w_G.  Pinned by:
  * structure: the mixture reaches half its peak exactly at G/2, and its area is w_L + w_G
    (1 for Thompson and Olivero; within 0.73 % of 1 for Liu-Lin, whose weights do not sum to 1);
  * limits: a vanishing Lorentz width gives the Doppler Gaussian, a vanishing Doppler width the
    Lorentzian;
  * the widths against the exact Voigt full width found by root-finding on SciPy's voigt_profile:
    Olivero-Longbothum's formula to its quoted ~0.02 % (2.4e-4 measured over width ratios
    1e-3 .. 1e3), Liu-Lin's to 1.1e-4, Thompson's to 0.43 %;
  * the whole profile against SciPy's Voigt, relative to the Voigt's peak: 1.27 % (Thompson),
    1.34 % (Olivero), 0.64 % (Liu-Lin), the measured maxima over the same ratios;
  * the three independent parametrisations against each other at equal Gaussian and Lorentzian
    widths, where Liu-Lin's width equals Olivero's and Liu-Lin's Lorentz weight equals the
    Thompson mixing of Olivero's width.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special

import oracle

LN2 = math.log(2.0)
KINDS = ["pv_thompson", "pv_olivero", "pv_liulin"]
RATIOS = np.logspace(-3, 3, 25)


def _voigt_fwhm(a, g):
    s = a / math.sqrt(2 * LN2)
    v0 = special.voigt_profile(0.0, s, g)
    return 2 * optimize.brentq(lambda x: special.voigt_profile(x, s, g) - 0.5 * v0, 0.0, 10 * (a + g) + 1.0,
                               xtol=1e-14, rtol=1e-14)


@pytest.mark.parametrize("kind", KINDS)
def test_half_maximum_at_half_the_common_width_and_area(kind):
    for rho in (1e-2, 0.3, 1.0, 4.0, 100.0):
        a, g = 0.7, 0.7 * rho
        G, wl, wg = oracle.pv_params(kind, a, g)
        f = oracle.profile(kind, np.array([0.0, G[0] / 2, -G[0] / 2]), a, g)
        assert f[1] / f[0] == pytest.approx(0.5, rel=1e-13) and f[2] / f[0] == pytest.approx(0.5, rel=1e-13)
        area = integrate.quad(lambda x: oracle.profile(kind, np.array([x]), a, g)[0], -np.inf, np.inf,
                              limit=400, epsabs=0, epsrel=1e-11)[0]
        assert area == pytest.approx(wl[0] + wg[0], rel=1e-8)
        if kind == "pv_liulin":
            assert abs(area - 1.0) < 7.3e-3
        else:
            assert area == pytest.approx(1.0, rel=1e-8)


@pytest.mark.parametrize("kind", KINDS)
def test_gaussian_and_lorentzian_limits(kind):
    x = np.linspace(-3.0, 3.0, 61)
    a = 0.4
    gauss = oracle.profile("gauss_hwhm", x, a)
    pv = oracle.profile(kind, x, a, 0.0)
    if kind == "pv_liulin":  # weights 0.99857 / 0.00079 at the Gaussian end: within 2e-3 of the peak
        assert np.max(np.abs(pv - gauss)) / gauss.max() < 2e-3
    else:
        assert np.max(np.abs(pv - gauss) / gauss) < 1e-13
    g = 0.25
    lor = oracle.profile("lorentz", x, 0.0, g)
    pv = oracle.profile(kind, x, 0.0, g)
    if kind == "pv_liulin":  # weights 0.99529 / 0.00425 at the Lorentzian end
        assert np.max(np.abs(pv - lor)) / lor.max() < 5e-3
    else:
        assert np.max(np.abs(pv - lor) / lor) < 2e-5


@pytest.mark.parametrize("kind,bound", [("pv_olivero", 2.5e-4), ("pv_liulin", 1.2e-4), ("pv_thompson", 4.5e-3)])
def test_width_against_the_exact_voigt_full_width(kind, bound):
    worst = 0.0
    for rho in RATIOS:
        a, g = 1.0, float(rho)
        G, _, _ = oracle.pv_params(kind, a, g)
        worst = max(worst, abs(G[0] - _voigt_fwhm(a, g)) / _voigt_fwhm(a, g))
    assert worst <= bound, worst
    assert worst > bound / 20  # the formula is an approximation, not the exact width


@pytest.mark.parametrize("kind,bound", [("pv_thompson", 1.3e-2), ("pv_olivero", 1.4e-2), ("pv_liulin", 6.5e-3)])
def test_profile_against_scipy_voigt(kind, bound):
    worst = 0.0
    for rho in RATIOS:
        a, g = 1.0, float(rho)
        s = a / math.sqrt(2 * LN2)
        x = np.linspace(-30 * (a + g), 30 * (a + g), 60001)
        v = special.voigt_profile(x, s, g)
        pv = oracle.profile(kind, x, a, g)
        worst = max(worst, float(np.max(np.abs(pv - v)) / v.max()))
    assert worst <= bound, worst


def test_parametrisations_agree_at_equal_widths():
    a = g = 0.9
    Go, wlo, _ = oracle.pv_params("pv_olivero", a, g)
    Gl, wll, wgl = oracle.pv_params("pv_liulin", a, g)
    assert Gl[0] == pytest.approx(Go[0], rel=1e-4)
    assert wll[0] == pytest.approx(wlo[0], abs=5e-4)
    assert wll[0] == pytest.approx(0.68188, abs=1e-12) and wgl[0] == pytest.approx(0.32460, abs=1e-12)
    # Olivero's width at equal widths, 0.5346 + sqrt(1.2166), in units of the full widths
    assert Go[0] / (2 * a) == pytest.approx(1.63759592, rel=1e-8)


@pytest.mark.parametrize("kind", KINDS)
def test_pseudo_voigt_cross_section_keeps_the_intensity(kind):
    # two lines on a fine grid with a wide cut-off: the summed sigma carries sum I (w_L + w_G)
    # less the Lorentzian wing beyond the cut-off
    E = np.array([0.0, 1000.0, 1003.0]); g = np.array([1, 3, 5], np.int32)
    up = np.array([1, 2], np.int32); lo = np.array([0, 0], np.int32); A = np.array([5.0, 9.0])
    gr = np.array([0.05, 0.08], np.float32); ne = np.array([0.5, 0.7], np.float32)
    cut, dnu = 200.0, 0.001
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind=kind, T=800.0, P=1.0, nu_min=700.0, dnu=dnu,
                   n_grid=700001, cut=cut)
    alpha, gamma = r["alpha"], r["gamma"]
    G, wl, wg = oracle.pv_params(kind, alpha, gamma)
    kept = r["I"] * (wl * (2 / math.pi) * np.arctan(cut / (G / 2)) + wg)
    assert r["sigma"].sum() * dnu == pytest.approx(kept.sum(), rel=2e-6)
