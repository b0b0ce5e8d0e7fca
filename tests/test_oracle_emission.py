"""Pins of the oracle's emission intensities, vibronic-density populations and
cooling function (Secs. 2.4.2 and 3) against physics that does not go through them:
Kirchhoff's law, closed-form cooling functions of a two-level system and of a
harmonic ladder, separable partition functions, and the reductions of the
density model to LTE and to the two-temperature model.
"""
import math

import numpy as np
import pytest

import oracle

C = 2.99792458e10
H = 6.62607015e-27
GRID = (0.0, 1.0, 40001)   # nu_min, dnu, n  (covers every line below)
CUT = 5.0


def _lines(E, g, up, lo, A, T, *, Tv=0.0, Ev=None, nv=None, emission=False, Q=None):
    if Q is None:
        if nv is not None:
            Q = oracle.partition_density(E, g, Ev, nv, T)[0]
        else:
            Q = oracle.partition(E, g, Ev if Tv > 0 else None, T, Tv)[0]
    nu, val, keep, _, _ = oracle.intensities(E, g, Ev, np.asarray(up, np.int32), np.asarray(lo, np.int32),
                                             np.asarray(A, np.float64), T, Tv, Q, *GRID, CUT, 0.0,
                                             emission=emission, n_vib=nv)
    return nu, val, keep.astype(bool), Q


def _random_levels(rng, n=60):
    E = np.sort(rng.uniform(0.0, 15000.0, n))
    g = rng.integers(1, 30, n).astype(np.int32)
    up = rng.integers(n // 2, n, 200)
    lo = rng.integers(0, n // 2, 200)
    A = 10.0 ** rng.uniform(-3, 2, 200)
    return E, g, up, lo, A


def test_kirchhoff_emission_over_absorption_is_planck():
    # In LTE, epsilon / I = 2 h c^2 nu^3 / (exp(c2 nu / T) - 1) (Planck's law per wavenumber,
    # per steradian): a dropped population factor, a wrong degeneracy or a lost nu fails it.
    rng = np.random.default_rng(7)
    E, g, up, lo, A = _random_levels(rng)
    for T in (500.0, 2500.0):
        nu, I, k1, _ = _lines(E, g, up, lo, A, T)
        _, eps, k2, _ = _lines(E, g, up, lo, A, T, emission=True)
        m = k1 & k2 & (nu > 0)
        assert m.sum() > 100
        planck = 2 * H * C ** 2 * nu[m] ** 3 / np.expm1(oracle.c2() * nu[m] / T)
        np.testing.assert_allclose(eps[m] / I[m], planck, rtol=1e-12)


def test_emission_einstein_route_single_line():
    # epsilon = (h c nu) A N_u / (4 pi), N_u = g' exp(-c2 E'/T) / Q: energy per photon times
    # the spontaneous rate of the upper-state population, per steradian.
    Eu, El, gu, A, T, Q = 4321.0, 1234.0, 7, 3.5, 1500.0, 87.0
    E = np.array([El, Eu]); g = np.array([1, gu], np.int32)
    nu, eps, keep, _ = _lines(E, g, [1], [0], [A], T, emission=True, Q=Q)
    ref = H * C * (Eu - El) * A * gu * math.exp(-oracle.c2() * Eu / T) / Q / (4 * math.pi)
    assert keep[0] and eps[0] == pytest.approx(ref, rel=1e-14)


def test_cooling_function_two_level_closed_form():
    # W = h c w A g1 x / (4 pi (g0 + g1 x)), x = exp(-c2 w / T)
    w, g0, g1, A = 2143.27, 1, 3, 33.0
    E = np.array([0.0, w]); g = np.array([g0, g1], np.int32)
    for T in (200.0, 1000.0, 5000.0):
        Q = oracle.partition(E, g, None, T)[0]
        W = oracle.cooling_function(E, g, None, np.array([1], np.int32), np.array([0], np.int32),
                                    np.array([A]), T, 0.0, Q)
        x = math.exp(-oracle.c2() * w / T)
        assert W == pytest.approx(H * C * w * A * g1 * x / (4 * math.pi * (g0 + g1 * x)), rel=1e-13)


def test_cooling_function_harmonic_ladder_mean_quantum_number():
    # Levels E = w v (g = 1, v = 0..N), lines v -> v-1 with A_v = v A1 (harmonic oscillator):
    # W = (h c w A1 / 4 pi) <v>, <v> = sum v x^v / sum x^v (closed form of the truncated ladder).
    w, A1, N = 1580.0, 2.0, 60
    v = np.arange(N + 1)
    E = w * v
    g = np.ones(N + 1, np.int32)
    up = v[1:].astype(np.int32); lo = (v[1:] - 1).astype(np.int32)
    A = A1 * v[1:].astype(np.float64)
    for T in (800.0, 3000.0, 20000.0):
        x = math.exp(-oracle.c2() * w / T)
        mean_v = x * (1 - (N + 1) * x ** N + N * x ** (N + 1)) / ((1 - x) * (1 - x ** (N + 1)))
        Q = oracle.partition(E, g, None, T)[0]
        W = oracle.cooling_function(E, g, None, up, lo, A, T, 0.0, Q)
        assert W == pytest.approx(H * C * w * A1 * mean_v / (4 * math.pi), rel=1e-12)


def test_cooling_function_is_the_sum_of_emission_intensities_and_skips_negative_nu():
    rng = np.random.default_rng(11)
    E, g, up, lo, A = _random_levels(rng)
    up2 = np.concatenate([up, lo[:20]]); lo2 = np.concatenate([lo, up[:20]])   # 20 lines with nu < 0
    A2 = np.concatenate([A, A[:20]])
    T = 1700.0
    Q = oracle.partition(E, g, None, T)[0]
    W = oracle.cooling_function(E, g, None, up2.astype(np.int32), lo2.astype(np.int32), A2, T, 0.0, Q)
    nu = E[up2] - E[lo2]
    brute = sum(H * C * A2[i] * nu[i] * g[up2[i]] * math.exp(-oracle.c2() * E[up2[i]] / T) / (4 * math.pi * Q)
                for i in range(nu.size) if nu[i] > 0)
    assert W == pytest.approx(brute, rel=1e-13)


# --------------------------------------------------------------------------- vibronic densities

def _manifolds(nv_levels=4, nJ=120):
    """Separable levels E = E_vib(v) + B J(J+1), g = 2J+1, the same rotational ladder in
    every vibrational manifold."""
    ev = 2143.0 * np.arange(nv_levels) - 13.0 * np.arange(nv_levels) ** 2
    J = np.arange(nJ)
    er = 1.93 * J * (J + 1.0)
    E = (ev[:, None] + er[None, :]).ravel()
    Ev = np.repeat(ev, nJ)
    g = np.tile((2 * J + 1).astype(np.int32), nv_levels)
    return ev, er, J, E, Ev, g


def test_density_partition_separable_closed_form():
    # with the same rotational ladder in every manifold and sum n_v = 1, Eq. (Q nlte Nvib)
    # gives Q = Q_rot(T_rot) whatever the densities
    ev, er, J, E, Ev, g = _manifolds()
    dens = np.array([0.55, 0.25, 0.15, 0.05])
    nv = np.repeat(dens, J.size)
    for Tr in (300.0, 1500.0):
        Q = oracle.partition_density(E, g, Ev, nv, Tr)[0]
        Qr = oracle.partition(er, (2 * J + 1).astype(np.int32), None, Tr)[0]
        assert Q == pytest.approx(Qr, rel=1e-13)


def test_density_with_boltzmann_densities_is_lte():
    # n_v proportional to exp(-c2 E_vib / T) and T_rot = T: populations, Q and the stimulated
    # emission factor all become the LTE ones (absorption and emission).
    ev, er, J, E, Ev, g = _manifolds()
    T = 1800.0
    nv = np.exp(-oracle.c2() * Ev / T)
    rng = np.random.default_rng(3)
    up = rng.integers(0, E.size, 300); lo = rng.integers(0, E.size, 300)
    A = 10.0 ** rng.uniform(-2, 2, 300)
    for emission in (False, True):
        _, a, ka, _ = _lines(E, g, up, lo, A, T, emission=emission)
        _, d, kd, _ = _lines(E, g, up, lo, A, T, Ev=Ev, nv=nv, emission=emission)
        assert np.array_equal(ka, kd) and ka.sum() > 50
        np.testing.assert_allclose(d[kd], a[ka], rtol=1e-12)


def test_density_emission_with_boltzmann_densities_is_treanor_emission():
    # emission has no stimulated factor, so n_v ~ exp(-c2 E_vib / T_vib) reproduces the
    # two-temperature emission of Eq. (nlte em 2T) at any T_rot
    ev, er, J, E, Ev, g = _manifolds()
    Tv, Tr = 3200.0, 700.0
    nv = np.exp(-oracle.c2() * Ev / Tv)
    rng = np.random.default_rng(5)
    up = rng.integers(0, E.size, 300); lo = rng.integers(0, E.size, 300)
    A = 10.0 ** rng.uniform(-2, 2, 300)
    _, t2, k2, _ = _lines(E, g, up, lo, A, Tr, Tv=Tv, Ev=Ev, emission=True)
    _, dd, kd, _ = _lines(E, g, up, lo, A, Tr, Ev=Ev, nv=nv, emission=True)
    assert np.array_equal(k2, kd) and k2.sum() > 50
    np.testing.assert_allclose(dd[kd], t2[k2], rtol=1e-12)


def test_density_absorption_single_line_and_scale_invariance():
    # Eq. (nlte ab pop density) on one line, and invariance under a common scale of n_v
    ev, er, J, E, Ev, g = _manifolds()
    dens = np.array([0.4, 0.3, 0.2, 0.1])
    nv = np.repeat(dens, J.size)
    Tr = 900.0
    l = 1 * J.size + 10          # v = 1, J = 10
    u = 2 * J.size + 11          # v = 2, J = 11
    _, I, keep, Q = _lines(E, g, [u], [l], [5.0], Tr, Ev=Ev, nv=nv)
    c2 = oracle.c2()
    nu = E[u] - E[l]
    ref = g[u] * 5.0 * dens[1] * math.exp(-c2 * er[10] / Tr) * (1 - math.exp(-c2 * nu / Tr)) / \
        (8 * math.pi * C * nu * nu * Q)
    assert keep[0] and I[0] == pytest.approx(ref, rel=1e-13)
    _, I7, _, _ = _lines(E, g, [u], [l], [5.0], Tr, Ev=Ev, nv=7.3 * nv)
    assert I7[0] == pytest.approx(I[0], rel=1e-14)
    # the paper's total population F (Eq. F nlte Nvib) sums to one over all states
    F = g * nv * np.exp(-c2 * (E - Ev) / Tr) / Q
    assert F.sum() == pytest.approx(1.0, rel=1e-13)


def test_density_model_argument_errors():
    ev, er, J, E, Ev, g = _manifolds(2, 5)
    nv = np.ones(E.size)
    with pytest.raises(oracle.OracleError):   # densities without E_vib
        oracle.partition_density(E, g, None, nv, 500.0)
    with pytest.raises(oracle.OracleError):   # densities and T_vib together are ambiguous
        oracle.intensities(E, g, Ev, np.array([3], np.int32), np.array([0], np.int32), np.array([1.0]),
                           500.0, 900.0, 1.0, *GRID, CUT, 0.0, n_vib=nv)
