"""Pins of the oracle's line widths and of its inverted-population (gain) branch.

Widths (Table profile; the formulas the paper takes from its predecessor):
  * the Doppler HWHM is derived here from the physics it stands for: the
    line-of-sight velocity distribution of a Maxwell gas, whose second moment is
    integrated numerically (no closed form typed in), turned into the Gaussian
    line shape of the Doppler-shifted centre and its half width; and checked
    against the spectroscopists' rule alpha_D = 3.581e-7 nu sqrt(T / M) cm^-1;
  * the pressure law gamma = gamma_ref (T_ref / T)^n P is pinned by its limits
    and its logarithmic derivatives (gamma = gamma_ref P at T = T_ref; linear in P;
    d ln gamma / d ln T = -n), which fail for a dropped P, an inverted
    temperature ratio or a wrong exponent sign.
Gain (Sec. 3.2-3.3, two-temperature populations): when T_vib > T_rot a line
whose upper state has more vibrational but less rotational energy than its lower
state can have a larger upper-level population per degeneracy than lower, and its
absorption intensity is negative.  Such lines are kept when |I| >= S_min and the
list exponent follows |I| (reading R10).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

C = 2.99792458e10
KB = 1.380649e-16
NA = 6.02214076e23


# --------------------------------------------------------------------------- Doppler width

def _doppler_hwhm_from_maxwell(nu, T, M):
    """HWHM of the Doppler profile of a line at nu for molecules of M g/mol at T, from the
    line-of-sight Maxwell distribution p(v) ~ exp(-m v^2 / (2 k T)) by quadrature."""
    m = M / NA                                   # g per molecule
    p = lambda v: math.exp(-m * v * v / (2.0 * KB * T))
    vmax = 40.0 * math.sqrt(KB * T / m) * 10.0   # far beyond the distribution's reach
    z = integrate.quad(p, -vmax, vmax, points=[0.0], limit=400, epsabs=0.0, epsrel=1e-13)[0]
    s2 = integrate.quad(lambda v: v * v * p(v), -vmax, vmax, points=[0.0], limit=400, epsabs=0.0,
                        epsrel=1e-13)[0] / z
    # a molecule moving at v along the line of sight absorbs at nu (1 + v / c): the line shape is
    # the velocity distribution mapped by d nu = nu v / c, a Gaussian of standard deviation
    # nu sigma_v / c, whose half width at half maximum is that times sqrt(2 ln 2)
    sd = nu * math.sqrt(s2) / C
    return sd * math.sqrt(2.0 * math.log(2.0))


@pytest.mark.parametrize("nu,T,M", [(2000.0, 296.0, 44.0), (5000.0, 1000.0, 18.0), (25000.0, 2000.0, 18.0),
                                    (300.0, 80.0, 2.0)])
def test_doppler_width_from_the_maxwell_velocity_distribution(nu, T, M):
    a, _ = oracle.widths("gauss_doppler", np.array([nu]), None, None, T, 1.0, mass_da=M)
    assert a[0] == pytest.approx(_doppler_hwhm_from_maxwell(nu, T, M), rel=1e-9)


def test_doppler_width_textbook_rule():
    # alpha_D [cm^-1] = 3.581e-7 nu sqrt(T / M), M in g/mol (the numerical form quoted in
    # spectroscopy texts and line-database documentation, four significant figures)
    for nu, T, M in [(2000.0, 296.0, 44.0), (1000.0, 1500.0, 18.0), (4300.0, 700.0, 16.0)]:
        a, _ = oracle.widths("voigt", np.array([nu]), np.array([0.05], np.float32), np.array([0.5], np.float32),
                             T, 1.0, mass_da=M)
        assert a[0] == pytest.approx(3.581e-7 * nu * math.sqrt(T / M), rel=2e-4)


def test_doppler_width_is_the_profile_half_width():
    # the Gaussian the oracle evaluates has its half maximum exactly alpha away from the centre
    nu, T, M = 3000.0, 900.0, 28.0
    a, _ = oracle.widths("gauss_doppler", np.array([nu]), None, None, T, 1.0, mass_da=M)
    f = oracle.profile("gauss_doppler", np.array([0.0, a[0], -a[0]]), a[0])
    assert f[1] / f[0] == pytest.approx(0.5, rel=1e-14) and f[2] / f[0] == pytest.approx(0.5, rel=1e-14)


# --------------------------------------------------------------------------- pressure law

def _gamma(gref, n, T, P, T_ref=296.0, kind="lorentz"):
    _, g = oracle.widths(kind, np.array([1000.0]), np.array([gref], np.float32), np.array([n], np.float32),
                         T, P, T_ref=T_ref)
    return g[0]


def test_pressure_width_at_the_reference_temperature_is_gamma_ref_times_P():
    gref = float(np.float32(0.0734))
    for P in (1e-5, 0.1, 1.0, 37.0):
        assert _gamma(gref, 0.63, 296.0, P) == pytest.approx(gref * P, rel=1e-15)
    assert _gamma(gref, 0.63, 500.0, 0.0) == 0.0


def test_pressure_width_temperature_exponent_by_finite_differences():
    # d ln gamma / d ln T = -n (a wider line at low T for n > 0), d ln gamma / d ln P = 1
    gref, T, P, h = 0.05, 1234.0, 0.7, 1e-4
    for n in (0.25, 0.5, 0.75):
        n32 = float(np.float32(n))
        dlnT = (math.log(_gamma(gref, n, T * (1 + h), P)) - math.log(_gamma(gref, n, T * (1 - h), P))) / \
               (math.log(1 + h) - math.log(1 - h))
        assert dlnT == pytest.approx(-n32, rel=1e-8)
        dlnP = (math.log(_gamma(gref, n, T, P * (1 + h))) - math.log(_gamma(gref, n, T, P * (1 - h)))) / \
               (math.log(1 + h) - math.log(1 - h))
        assert dlnP == pytest.approx(1.0, rel=1e-10)
    assert _gamma(gref, 0.5, 300.0, 1.0) < _gamma(gref, 0.5, 296.0 / 2, 1.0)


def test_pressure_width_special_values_and_reference_temperature():
    # at T = 4 T_ref with n = 1/2 the width halves; another T_ref moves the law accordingly
    gref = float(np.float32(0.08))
    assert _gamma(gref, 0.5, 4 * 296.0, 2.0) == pytest.approx(gref * 2.0 / 2.0, rel=1e-14)
    assert _gamma(gref, 0.5, 4 * 250.0, 2.0, T_ref=250.0) == pytest.approx(gref, rel=1e-14)
    # the Doppler kinds carry no pressure width; the Voigt kind carries the same one as Lorentz
    assert _gamma(gref, 0.5, 1000.0, 1.0, kind="gauss_doppler") == 0.0
    assert _gamma(gref, 0.5, 1000.0, 1.0, kind="voigt") == _gamma(gref, 0.5, 1000.0, 1.0, kind="lorentz")


# --------------------------------------------------------------------------- gain (inverted populations)

def _inverted_list():
    """Two-temperature levels: state 0 (E_vib 0, E_rot 800), state 1 (E_vib 2000, E_rot 0),
    state 2 (E_vib 2000, E_rot 30), state 3 (E_vib 0, E_rot 0)."""
    Ev = np.array([0.0, 2000.0, 2000.0, 0.0])
    Er = np.array([800.0, 0.0, 30.0, 0.0])
    E = Ev + Er
    g = np.array([3, 5, 7, 1], np.int32)
    up = np.array([1, 2, 1], np.int32)      # 0 -> 1 (inverted), 0 -> 2 (inverted), 3 -> 1 (normal)
    lo = np.array([0, 0, 3], np.int32)
    A = np.array([2.0, 40.0, 1.5])
    return E, g, Ev, up, lo, A


def test_inverted_line_has_negative_intensity_equal_to_the_population_difference():
    E, g, Ev, up, lo, A = _inverted_list()
    Tr, Tv = 300.0, 6000.0
    c2 = oracle.c2()
    Q = oracle.partition(E, g, Ev, Tr, Tv)[0]
    nu, I, keep, _, _ = oracle.line_intensities(E, g, Ev, up, lo, A, Tr, Tv, Q, 0.0, 0.01, 10 ** 7, 25.0)
    for t in range(up.size):
        u, l = up[t], lo[t]
        # absorption minus stimulated emission from the level populations per degeneracy:
        # I = g' A / (8 pi c nu^2) (n''/g'' - n'/g') with n/g = exp(-c2 E_vib/T_vib - c2 E_rot/T_rot) / Q
        pl = math.exp(-c2 * Ev[l] / Tv - c2 * (E[l] - Ev[l]) / Tr) / Q
        pu = math.exp(-c2 * Ev[u] / Tv - c2 * (E[u] - Ev[u]) / Tr) / Q
        ref = g[u] * A[t] / (8 * math.pi * C * nu[t] ** 2) * (pl - pu)
        assert I[t] == pytest.approx(ref, rel=1e-12)
    assert I[0] < 0 and I[1] < 0 and I[2] > 0, I
    assert keep.all()


def test_inverted_lines_keep_rule_and_exponent_follow_the_magnitude():
    E, g, Ev, up, lo, A = _inverted_list()
    Tr, Tv = 300.0, 6000.0
    Q = oracle.partition(E, g, Ev, Tr, Tv)[0]
    args = (E, g, Ev, up, lo, A, Tr, Tv, Q, 0.0, 0.01, 10 ** 7, 25.0)
    _, I, keep, _, _ = oracle.line_intensities(*args)
    big = int(np.argmax(np.abs(I)))
    assert I[big] < 0, "the fixture's strongest line is an inverted one"
    # threshold between the magnitudes of the two inverted lines: the weaker one goes, the other stays
    thr = math.sqrt(abs(I[0]) * abs(I[1]))
    _, I2, keep2, _, _ = oracle.line_intensities(*args, thr)
    weak, strong = (0, 1) if abs(I[0]) < abs(I[1]) else (1, 0)
    assert not keep2[weak] and keep2[strong] and I2[strong] < 0
    # the keep rule is on |I|: exactly at |I| the line is kept, just above it is dropped
    assert oracle.line_intensities(*args, abs(I[strong]))[2][strong]
    assert not oracle.line_intensities(*args, abs(I[strong]) * (1 + 1e-12))[2][strong]
    # the list exponent is that of the largest |I|, here a negative intensity
    k = oracle.list_exponent(I, keep)
    assert k == math.frexp(abs(I[big]))[1]
    Is = oracle.scale_intensities(I, keep, k)
    assert Is[big] < 0 and 0.5 <= abs(float(Is[big])) < 1.0


def test_inverted_line_becomes_normal_in_lte():
    E, g, Ev, up, lo, A = _inverted_list()
    Q = oracle.partition(E, g, None, 300.0)[0]
    _, I, keep, _, _ = oracle.line_intensities(E, g, None, up, lo, A, 300.0, 0.0, Q, 0.0, 0.01, 10 ** 7, 25.0)
    assert (I[keep.astype(bool)] > 0).all()


def test_inverted_line_enters_sigma_with_its_sign():
    E, g, Ev, up, lo, A = _inverted_list()
    gr = np.full(3, 0.05, np.float32); ne = np.full(3, 0.5, np.float32)
    r = oracle.run(E, g, Ev, up[:1], lo[:1], A[:1], gr[:1], ne[:1], kind="voigt", T=300.0, T_vib=6000.0, P=1.0,
                   nu_min=1150.0, dnu=0.01, n_grid=10001, cut=5.0)
    assert r["I"][0] < 0
    s = r["sigma"]
    assert s.max() <= 0.0 and s.min() < 0.0
    area = s.sum() * 0.01
    # the sampled profile over a 10-cm^-1 window of a line ~0.1 cm^-1 wide keeps most of the area
    assert area == pytest.approx(r["I"][0], rel=0.02)
