"""Pins of the FP64 oracle against things other than itself.

Each test fixes a part of the oracle by a closed form, an invariant, an
independent implementation (SciPy's Faddeeva / Voigt, the Einstein-coefficient
route to a line intensity) or brute force on tiny inputs, chosen so that a
dropped term, a wrong sign or index, or a transposed operand fails one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import synth

C = 2.99792458e10
H = 6.62607015e-27
KB = 1.380649e-16
NA = 6.02214076e23
LN2 = math.log(2.0)


# --------------------------------------------------------------------------- constants

def test_c2_value():
    # c2 = hc/k_B = 1.438776877... cm K (CODATA 2018, exact inputs)
    assert oracle.c2() == pytest.approx(1.4387768775039337, rel=1e-15)


# --------------------------------------------------------------------------- Faddeeva / profiles

def test_faddeeva_matches_scipy_wofz():
    x = np.concatenate([-np.logspace(-4, 4, 60), np.logspace(-4, 4, 60), np.linspace(0, 10, 101)])
    for y in np.concatenate([[0.0], np.logspace(-4, 4, 25)]):
        w = oracle.faddeeva(x, y)
        ref = special.wofz(x + 1j * y)
        rel = np.abs(w - ref) / np.abs(ref)
        assert rel.max() < 1e-12, (y, rel.max())
        if y >= 1e-4:
            relre = np.abs(w.real - ref.real) / np.abs(ref.real)
            assert relre.max() < 1e-10, (y, relre.max())


def test_voigt_matches_scipy_voigt_profile():
    # log grid of (x/s, gamma/s) in [1e-4, 1e4]^2, as in the paper's SciPy Voigt reference
    for s in (0.01, 1.0):
        alpha = s * math.sqrt(2 * LN2)
        for gs in np.logspace(-4, 4, 9):
            gamma = gs * s
            x = s * np.concatenate([np.logspace(-4, 4, 41), -np.logspace(-4, 4, 41)])
            f = oracle.profile("voigt", x, alpha, gamma)
            ref = special.voigt_profile(x, s, gamma)
            assert np.max(np.abs(f - ref) / ref) < 1e-10


def test_voigt_centre_erfcx_closed_form():
    for alpha, gamma in [(0.02, 0.001), (0.01, 0.05), (1.0, 1.0), (0.3, 30.0)]:
        s = alpha / math.sqrt(2 * LN2)
        v0 = special.erfcx(gamma / (s * math.sqrt(2))) / (s * math.sqrt(2 * math.pi))
        assert oracle.profile("voigt", np.array([0.0]), alpha, gamma)[0] == pytest.approx(v0, rel=1e-12)


def test_voigt_limits():
    x = np.linspace(-0.1, 0.1, 201)
    a = 0.02
    g = oracle.profile("gauss_hwhm", x, a)
    v = oracle.profile("voigt", x, a, 1e-9)
    assert np.max(np.abs(v - g)) / g.max() < 1e-6
    gam = 0.05
    lor = oracle.profile("lorentz", x, 0.0, gam)
    v = oracle.profile("voigt", x, 1e-7, gam)
    assert np.max(np.abs(v - lor) / lor) < 1e-6


def test_gauss_half_width_and_peak():
    # HWHM means f(alpha) = f(0)/2; unit area fixes f(0) = sqrt(ln2/pi)/alpha
    a = 0.037
    f0, fa = oracle.profile("gauss_hwhm", np.array([0.0, a]), a)
    assert fa / f0 == pytest.approx(0.5, rel=1e-14)
    lo0, loa = oracle.profile("lorentz", np.array([0.0, a]), 0.0, a)
    assert loa / lo0 == pytest.approx(0.5, rel=1e-14)
    assert lo0 == pytest.approx(1.0 / (math.pi * a), rel=1e-14)


@pytest.mark.parametrize("kind", ["gauss_hwhm", "lorentz", "voigt"])
def test_truncated_profile_integrals(kind):
    # int_{-c}^{c} G = erf(c sqrt(ln2)/alpha); int L = (2/pi) atan(c/gamma); the
    # Voigt integral by adaptive quadrature of SciPy's voigt_profile.
    a, gm, cut = 0.05, 0.03, 1.5
    if kind == "gauss_hwhm":
        exact = math.erf(cut * math.sqrt(LN2) / a)
    elif kind == "lorentz":
        exact = 2 / math.pi * math.atan(cut / gm)
    else:
        s = a / math.sqrt(2 * LN2)
        exact = 2 * integrate.quad(lambda t: special.voigt_profile(t, s, gm), 0, cut,
                                   points=[0.1, 0.5], limit=500, epsabs=0, epsrel=1e-13)[0]
    x = np.linspace(-cut, cut, 600_001)
    f = oracle.profile(kind, x, a, gm)
    num = integrate.simpson(f, x=x)
    assert num == pytest.approx(exact, rel=1e-9)


@pytest.mark.parametrize("kind", ["gauss_hwhm", "lorentz", "voigt"])
def test_profile_width_derivatives(kind):
    x = np.linspace(-0.4, 0.4, 41)
    a, g = 0.03, 0.02
    f, fa, fg = oracle.profile(kind, x, a, g, derivs=True)
    h = 1e-6
    fa_fd = (oracle.profile(kind, x, a * (1 + h), g) - oracle.profile(kind, x, a * (1 - h), g)) / (2 * a * h)
    assert np.allclose(fa, fa_fd, rtol=1e-6, atol=1e-8 * np.abs(f).max())
    if kind != "gauss_hwhm":
        fg_fd = (oracle.profile(kind, x, a, g * (1 + h)) - oracle.profile(kind, x, a, g * (1 - h))) / (2 * g * h)
        assert np.allclose(fg, fg_fd, rtol=1e-6, atol=1e-8 * np.abs(f).max())


# --------------------------------------------------------------------------- partition functions

def test_partition_harmonic_closed_form():
    # E = omega v, g = 1, v = 0..N: Q = (1 - x^{N+1})/(1 - x), x = exp(-c2 omega / T)
    om, N, T = 1234.5, 40, 1700.0
    E = om * np.arange(N + 1)
    x = math.exp(-oracle.c2() * om / T)
    Q = oracle.partition(E, np.ones(N + 1, np.int32), None, T)[0]
    assert Q == pytest.approx((1 - x ** (N + 1)) / (1 - x), rel=1e-14)


def test_partition_rigid_rotor_mulholland():
    # E = B J(J+1), g = 2J+1: Q ~ (T/th)(1 + th/3T + th^2/15T^2 + 4 th^3/315T^3), th = c2 B
    B, T = 1.9, 3000.0
    J = np.arange(0, 4000)
    Q = oracle.partition(B * J * (J + 1.0), (2 * J + 1).astype(np.int32), None, T)[0]
    th = oracle.c2() * B
    r = th / T
    assert Q == pytest.approx((1 / r) * (1 + r / 3 + r * r / 15 + 4 * r ** 3 / 315), rel=1e-9)


def test_partition_two_temperature_factorises():
    # separable levels E = E_vib(v) + E_rot(J): Q(T_vib, T_rot) = Q_vib(T_vib) Q_rot(T_rot)
    ev = np.array([0.0, 2143.0, 4260.0, 6350.0])
    J = np.arange(0, 300)
    er = 1.93 * J * (J + 1.0)
    gr = (2 * J + 1).astype(np.int32)
    E = (ev[:, None] + er[None, :]).ravel()
    Ev = np.repeat(ev, J.size)
    g = np.tile(gr, ev.size)
    Tv, Tr = 2500.0, 900.0
    Q2 = oracle.partition(E, g, Ev, Tr, Tv)[0]
    Qv = oracle.partition(ev, np.ones(4, np.int32), None, Tv)[0]
    Qr = oracle.partition(er, gr, None, Tr)[0]
    assert Q2 == pytest.approx(Qv * Qr, rel=1e-13)
    # and the two-temperature form at T_vib = T_rot is the LTE sum
    assert oracle.partition(E, g, Ev, 1300.0, 1300.0)[0] == pytest.approx(
        oracle.partition(E, g, None, 1300.0)[0], rel=1e-13)


def test_partition_derivatives_and_absent_states():
    E = np.array([0.0, 100.0, np.nan, 2500.0])
    g = np.array([1, 3, 5, 7], np.int32)
    T = 700.0
    Q, dQ, _ = oracle.partition(E, g, None, T)
    assert Q == pytest.approx(oracle.partition(E[[0, 1, 3]], g[[0, 1, 3]], None, T)[0], rel=1e-15)
    h = 1e-3
    fd = (oracle.partition(E, g, None, T + h)[0] - oracle.partition(E, g, None, T - h)[0]) / (2 * h)
    assert dQ == pytest.approx(fd, rel=1e-7)
    Ev = np.array([0.0, 0.0, 0.0, 2000.0])
    Q2, dQr, dQv = oracle.partition(E, g, Ev, T, 1500.0)
    fdr = (oracle.partition(E, g, Ev, T + h, 1500.0)[0] - oracle.partition(E, g, Ev, T - h, 1500.0)[0]) / (2 * h)
    fdv = (oracle.partition(E, g, Ev, T, 1500.0 + h)[0] - oracle.partition(E, g, Ev, T, 1500.0 - h)[0]) / (2 * h)
    assert dQr == pytest.approx(fdr, rel=1e-7) and dQv == pytest.approx(fdv, rel=1e-7)


def test_partition_overflow_is_an_error():
    with pytest.raises(oracle.OracleError) as e:
        oracle.partition(np.array([0.0, -1e6]), np.array([1, 1], np.int32), None, 300.0)
    assert e.value.code == 4


# --------------------------------------------------------------------------- intensities

def _one_line(Eu, El, gu, A, T, Tv=0.0, Evu=0.0, Evl=0.0, Q=1.0, grid=(0.0, 0.01, 10**7), cut=25.0, thr=0.0):
    E = np.array([El, Eu]); g = np.array([1, gu], np.int32); Ev = np.array([Evl, Evu])
    nu, I, keep, lo, hi = oracle.line_intensities(E, g, Ev, np.array([1], np.int32), np.array([0], np.int32),
                                                  np.array([A]), T, Tv, Q, grid[0], grid[1], grid[2], cut, thr)
    return nu[0], I[0], keep[0]


def test_intensity_einstein_coefficient_route():
    # Independent route through the Einstein B coefficients in frequency units:
    # B21 = c^3 A / (8 pi h f^3), g1 B12 = g2 B21, and the frequency-integrated
    # absorption per molecule (h f / c) B12 n1/N (1 - e^{-h f / k T}), divided by c
    # to integrate over wavenumber.  Lower-state population n1/N = g1 e^{-E1/kT}/Q.
    El, Eu, gu, gl, A, T, Q = 1200.0, 3456.75, 9, 7, 12.5, 1800.0, 345.6
    f = C * (Eu - El)                      # Hz
    E1 = H * C * El                        # erg
    B21 = C ** 3 * A / (8 * math.pi * H * f ** 3)
    B12 = gu / gl * B21
    pop = gl * math.exp(-E1 / (KB * T)) / Q
    ref = (H * f / C) * B12 * pop * (1 - math.exp(-H * f / (KB * T))) / C
    nu, I, keep = _one_line(Eu, El, gu, A, T, Q=Q)
    assert keep and nu == Eu - El
    assert I == pytest.approx(ref, rel=1e-13)


def test_intensity_two_temperature_reduces_to_lte():
    for T in (300.0, 1900.0):
        a = _one_line(5000.0, 1400.0, 5, 3.0, T, Q=10.0)[1]
        b = _one_line(5000.0, 1400.0, 5, 3.0, T, Tv=T, Evu=4100.0, Evl=1000.0, Q=10.0)[1]
        assert b == pytest.approx(a, rel=1e-14)


def test_intensity_two_temperature_separates_vib_and_rot():
    # Raising T_vib multiplies a line's lower-state population by exp(c2 E''_vib (1/T1 - 1/T2))
    # and changes only the vibrational part of the stimulated-emission exponent.
    c2 = oracle.c2()
    Evl, Erl, Evu, Eru, Tr = 2000.0, 300.0, 4000.0, 320.0, 800.0
    I1 = _one_line(Evu + Eru, Evl + Erl, 3, 1.0, Tr, Tv=1500.0, Evu=Evu, Evl=Evl)[1]
    I2 = _one_line(Evu + Eru, Evl + Erl, 3, 1.0, Tr, Tv=3000.0, Evu=Evu, Evl=Evl)[1]
    pop = math.exp(-c2 * Evl / 3000.0) / math.exp(-c2 * Evl / 1500.0)
    se = (1 - math.exp(-c2 * ((Evu - Evl) / 3000.0 + (Eru - Erl) / Tr))) / \
         (1 - math.exp(-c2 * ((Evu - Evl) / 1500.0 + (Eru - Erl) / Tr)))
    assert I2 / I1 == pytest.approx(pop * se, rel=1e-13)


def test_intensity_linear_in_A_and_upper_degeneracy():
    b = _one_line(3000.0, 100.0, 4, 2.0, 1000.0)[1]
    assert _one_line(3000.0, 100.0, 4, 6.0, 1000.0)[1] == pytest.approx(3 * b, rel=1e-15)
    assert _one_line(3000.0, 100.0, 8, 2.0, 1000.0)[1] == pytest.approx(2 * b, rel=1e-15)


def test_drop_rules_and_errors():
    assert not _one_line(100.0, 300.0, 1, 1.0, 300.0)[2]           # nu < 0 discarded
    assert not _one_line(300.0, 300.0, 1, 1.0, 300.0)[2]           # nu = 0 discarded
    assert not _one_line(np.nan, 300.0, 1, 1.0, 300.0)[2]          # absent state
    assert not _one_line(5000.0, 0.0, 1, 1.0, 300.0, grid=(0.0, 1.0, 100))[2]   # window off-grid
    assert _one_line(123.9, 0.0, 1, 1.0, 300.0, grid=(0.0, 1.0, 100))[2]        # wing reaches the grid
    thr_I = _one_line(1000.0, 0.0, 1, 1.0, 300.0)[1]
    assert _one_line(1000.0, 0.0, 1, 1.0, 300.0, thr=thr_I)[2]
    assert not _one_line(1000.0, 0.0, 1, 1.0, 300.0, thr=thr_I * (1 + 1e-12))[2]
    E = np.array([0.0, 10.0]); g = np.array([1, 1], np.int32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.line_intensities(E, g, None, np.array([2], np.int32), np.array([0], np.int32), np.array([1.0]),
                                300.0, 0.0, 1.0, 0.0, 0.01, 100, 1.0)
    assert e.value.code == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.line_intensities(E, g, None, np.array([1], np.int32), np.array([0], np.int32), np.array([np.inf]),
                                300.0, 0.0, 1.0, 0.0, 0.01, 100, 1.0)
    assert e.value.code == 3


def test_literal_level_formula_overflows():
    # The unclamped quartic turns the energies hugely negative at high J; the
    # Boltzmann exponent then exceeds the double range and must be an error.
    w = synth.workload("doppler_1e5")
    E, g, Ev = w.states(literal=True)
    with pytest.raises(oracle.OracleError) as e:
        oracle.partition(E, g, None, w.T)
    assert e.value.code == 4


# --------------------------------------------------------------------------- windows, order, segments

def test_window_matches_brute_force_distance():
    rng = np.random.default_rng(3)
    nu_min, dnu, ng, cut = 10.0, 0.01, 5000, 0.37
    grid = nu_min + np.arange(ng) * dnu
    nus = rng.uniform(9.0, 61.0, 400)
    E = np.concatenate([[0.0], nus]); g = np.ones(E.size, np.int32)
    up = np.arange(1, E.size, dtype=np.int32); lo = np.zeros(nus.size, np.int32)
    nu, I, keep, ilo, ihi = oracle.line_intensities(E, g, None, up, lo, np.ones(nus.size), 500.0, 0.0, 1.0,
                                                    nu_min, dnu, ng, cut)
    for t in range(nus.size):
        d = np.abs(grid - nu[t])
        inside = np.nonzero(d <= cut)[0]
        near = np.abs(d - cut) < 1e-9
        if near.any():
            continue
        if inside.size == 0:
            assert not keep[t]
        else:
            assert keep[t] and ilo[t] == inside[0] and ihi[t] == inside[-1]


def test_sorted_order_is_lexicographic():
    rng = np.random.default_rng(5)
    nu = rng.choice(np.array([1.5, 2.25, 2.25, 3.0, 7.125]), 500)
    keep = (rng.random(500) < 0.8).astype(np.uint8)
    perm = oracle.sorted_order(nu, keep)
    idx = np.nonzero(keep)[0]
    ref = idx[np.lexsort((idx, nu[idx]))]
    assert np.array_equal(perm, ref)


def test_segment_ranges_brute_force():
    rng = np.random.default_rng(9)
    ilo = np.sort(rng.integers(0, 900, 300)); ihi = ilo + rng.integers(0, 40, 300)
    order = np.argsort(ilo, kind="stable")
    ilo, ihi = ilo[order], np.maximum.accumulate(ihi[order])
    first, last = oracle.segment_ranges(ilo, ihi, 1000, 64)
    for s in range(first.size):
        hit = np.nonzero((ihi >= 64 * s) & (ilo <= 64 * s + 63))[0]
        if hit.size:
            assert first[s] == hit[0] and last[s] == hit[-1] + 1
        else:
            assert first[s] == last[s]


def test_list_exponent_and_scaling():
    I = np.array([0.0, 3e-52, 7.5e-51, 1e-60])
    keep = np.array([1, 1, 1, 1], np.uint8)
    k = oracle.list_exponent(I, keep)
    assert 2.0 ** (k - 1) <= 7.5e-51 < 2.0 ** k
    Is = oracle.scale_intensities(I, keep, k)
    assert Is.dtype == np.float32 and Is.max() < 1.0 and Is[2] >= 0.5
    assert Is[1] == np.float32(3e-52 * 2.0 ** -k)


# --------------------------------------------------------------------------- cross sections

def _tiny_list(seed=11, n=40, nu_lo=5.0, nu_hi=15.0):
    rng = np.random.default_rng(seed)
    nus = rng.uniform(nu_lo, nu_hi, n)
    E = np.concatenate([[0.0], nus]); g = rng.integers(1, 10, E.size).astype(np.int32)
    up = np.arange(1, E.size, dtype=np.int32); lo = np.zeros(n, np.int32)
    A = 10 ** rng.uniform(-2, 2, n)
    gr = rng.uniform(0.03, 0.1, n).astype(np.float32); ne = rng.uniform(0.4, 0.8, n).astype(np.float32)
    return E, g, up, lo, A, gr, ne


@pytest.mark.parametrize("kind", ["gauss_doppler", "gauss_hwhm", "lorentz", "voigt"])
def test_cross_section_brute_force(kind):
    E, g, up, lo, A, gr, ne = _tiny_list()
    nu_min, dnu, ng, cut = 4.0, 0.005, 2400, 1.0
    T, P, M = 900.0, 0.7, 18.0
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind=kind, T=T, P=P, mass_da=M, hwhm=0.04,
                   nu_min=nu_min, dnu=dnu, n_grid=ng, cut=cut)
    grid = nu_min + np.arange(ng) * dnu
    ref = np.zeros(ng)
    Q = r["Q"][0]
    c2 = oracle.c2()
    for t in range(up.size):
        nu = E[up[t]] - E[lo[t]]
        I = g[up[t]] * A[t] / (8 * math.pi * C * nu ** 2) * math.exp(-c2 * E[lo[t]] / T) * \
            (1 - math.exp(-c2 * nu / T)) / Q
        x = grid - nu
        m = np.abs(x) <= cut
        alpha = nu / C * math.sqrt(2 * NA * KB * T * LN2 / M) if kind != "gauss_hwhm" else 0.04
        gamma = float(gr[t]) * (296.0 / T) ** float(ne[t]) * P
        s = alpha / math.sqrt(2 * LN2)
        if kind in ("gauss_doppler", "gauss_hwhm"):
            f = special.voigt_profile(x, s, 0.0)
        elif kind == "lorentz":
            f = special.voigt_profile(x, 0.0, gamma)
        else:
            f = special.voigt_profile(x, s, gamma)
        ref[m] += I * f[m]
    assert np.max(np.abs(r["sigma"] - ref)) <= 1e-10 * ref.max()


def test_cross_section_integral_equals_kept_intensity():
    # Fine grid (dnu << widths), wide grid: int sigma = sum_l I_l * (kept fraction),
    # the kept fraction of a Lorentzian truncated at cut being (2/pi) atan(cut/gamma).
    E, g, up, lo, A, gr, ne = _tiny_list(n=12, nu_lo=20.0, nu_hi=30.0)
    nu_min, dnu, ng, cut = 0.0, 0.001, 60_001, 2.0
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind="lorentz", T=500.0, P=1.0,
                   nu_min=nu_min, dnu=dnu, n_grid=ng, cut=cut)
    frac = 2 / math.pi * np.arctan(cut / r["gamma"])
    total = np.sum(r["I"] * frac)
    assert integrate.simpson(r["sigma"], dx=dnu) == pytest.approx(total, rel=1e-5)
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind="gauss_hwhm", hwhm=0.05, T=500.0,
                   nu_min=nu_min, dnu=dnu, n_grid=ng, cut=cut)
    assert integrate.simpson(r["sigma"], dx=dnu) == pytest.approx(r["I"].sum(), rel=1e-9)


def test_cross_section_permutation_invariant():
    E, g, up, lo, A, gr, ne = _tiny_list(n=60)
    kw = dict(kind="voigt", T=1200.0, P=0.3, nu_min=4.0, dnu=0.01, n_grid=1200, cut=1.5)
    a = oracle.run(E, g, None, up, lo, A, gr, ne, **kw)["sigma"]
    p = np.random.default_rng(1).permutation(up.size)
    b = oracle.run(E, g, None, up[p], lo[p], A[p], gr[p], ne[p], **kw)["sigma"]
    assert np.max(np.abs(a - b)) <= 1e-13 * a.max()


# --------------------------------------------------------------------------- adjoint

def _loss(params, base, w):
    E, g, Ev, up, lo, A, gr, ne, kw = base
    kw = dict(kw)
    kw.update(T=params["T"], T_vib=params["Tv"], P=params["P"])
    r = oracle.run(E, g, Ev, up, lo, params["A"], params["gr"], ne, **kw)
    return float(np.dot(w, r["sigma"])), r


@pytest.mark.parametrize("kind,Tv", [("voigt", 0.0), ("voigt", 2500.0), ("lorentz", 0.0), ("gauss_doppler", 0.0)])
def test_adjoint_matches_central_differences(kind, Tv):
    rng = np.random.default_rng(21)
    n = 25
    ev = np.array([0.0, 1800.0, 3550.0])
    J = np.arange(0, 30)
    E = (ev[:, None] + 0.9 * J * (J + 1.0)).ravel()
    Ev = np.repeat(ev, J.size)
    g = np.tile(2 * J + 1, 3).astype(np.int32)
    lo = rng.integers(0, J.size, n).astype(np.int32)
    up = (lo + J.size * rng.integers(1, 3, n)).astype(np.int32)
    A = 10 ** rng.uniform(-1, 1, n)
    gr = rng.uniform(0.03, 0.1, n).astype(np.float32); ne = rng.uniform(0.4, 0.8, n).astype(np.float32)
    nus = E[up] - E[lo]
    kw = dict(kind=kind, mass_da=18.0, nu_min=float(nus.min()) - 1.0, dnu=0.004,
              n_grid=int((nus.max() - nus.min() + 2.0) / 0.004), cut=0.8)
    base = (E, g, Ev, up, lo, A, gr, ne, kw)
    T, P = 1200.0, 0.5
    w = rng.standard_normal(kw["n_grid"])
    params = {"T": T, "Tv": Tv, "P": P, "A": A.copy(), "gr": gr.copy()}
    L0, r = _loss(params, base, w)
    gd = oracle.cross_section_grad(kind, E, Ev, up, lo, A, r["nu"], r["I"], r["alpha"], r["gamma"], ne,
                                   r["keep"], r["ilo"], r["ihi"], T, Tv, P, r["Q"], kw["nu_min"], kw["dnu"], w)

    def fd(key, h, idx=None):
        p1 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in params.items()}
        p2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in params.items()}
        if idx is None:
            p1[key] += h; p2[key] -= h
        else:
            p1[key][idx] += h; p2[key][idx] -= h
        return (_loss(p1, base, w)[0] - _loss(p2, base, w)[0]) / (2 * h)

    assert gd["dT"] == pytest.approx(fd("T", 1e-3 * T), rel=1e-5, abs=1e-7 * gd["dT_abs"])
    if kind in ("voigt", "lorentz"):
        assert gd["dP"] == pytest.approx(fd("P", 1e-4 * P), rel=1e-5, abs=1e-7 * gd["dP_abs"])
    if Tv > 0:
        assert gd["dTvib"] == pytest.approx(fd("Tv", 1e-3 * Tv), rel=1e-5, abs=1e-7 * gd["dTvib_abs"])
    for idx in (0, 7, 13):
        assert gd["dA"][idx] == pytest.approx(fd("A", 1e-6 * A[idx], idx), rel=1e-6, abs=1e-9 * np.abs(gd["dA"]).max())
        if kind in ("voigt", "lorentz"):
            # gamma_ref is float32 on input: step by a power of two so gamma_ref +- h are exact
            params["gr"] = params["gr"].astype(np.float64)
            assert gd["dgamma_ref"][idx] == pytest.approx(fd("gr", 2.0 ** -17, idx), rel=1e-5,
                                                          abs=1e-7 * np.abs(gd["dgamma_ref"]).max())
            params["gr"] = gr.copy()
