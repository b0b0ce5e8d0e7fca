"""Pins of the oracle's wavelength grids (Sec. 2.4.3; reading R21 in oracle/oracle.c).

A wavelength grid lambda_i = lambda_min + i dlambda (nm: U = 1e7, um: U = 1e4) samples sigma at
nu_i = U / lambda_i, with the cut-off in cm^-1.  Pinned by:
  * the window against brute force over every grid point of |U / lambda_i - nu| <= cut;
  * sigma on the wavelength grid against the pinned wavenumber path evaluated point by point at
    nu_i (a one-point wavenumber grid per lambda_i);
  * nm and um grids of the same points giving the same sigma;
  * the peak of an isolated narrow line at the grid point nearest U / nu;
  * the line order (descending nu, ties by index) keeping the windows monotone.
"""
import numpy as np
import pytest

import oracle

NM, UM = 1e7, 1e4


def _tiny(seed=3, n=60):
    rng = np.random.default_rng(seed)
    E = np.concatenate([[0.0], rng.uniform(200.0, 9000.0, 40)])
    g = rng.integers(1, 9, E.size).astype(np.int32)
    up = rng.integers(1, E.size, n).astype(np.int32)
    lo = np.zeros(n, np.int32)
    lo[: n // 3] = rng.integers(1, E.size, n // 3)
    A = 10.0 ** rng.uniform(-1, 2, n)
    gr = rng.uniform(0.03, 0.1, n).astype(np.float32)
    ne = rng.uniform(0.4, 0.8, n).astype(np.float32)
    return E, g, up, lo, A, gr, ne


def test_window_against_brute_force():
    rng = np.random.default_rng(1)
    lam0, dlam, n = 1000.0, 0.37, 40000          # 1000 .. 15800 nm: 10000 .. 633 cm^-1
    lam = lam0 + np.arange(n) * dlam
    nu_pts = NM / lam
    E = np.concatenate([[0.0], rng.uniform(100.0, 12000.0, 300), [10.0, 15.0]])
    g = np.ones(E.size, np.int32)
    up = np.arange(1, E.size, dtype=np.int32)
    lo = np.zeros(up.size, np.int32)
    A = np.ones(up.size)
    for cut in (5.0, 25.0):
        nu, I, keep, ilo, ihi = oracle.line_intensities(E, g, None, up, lo, A, 500.0, 0.0, 1.0, lam0, dlam, n, cut,
                                                        wl_unit=NM)
        for t in range(up.size):
            inside = np.nonzero(np.abs(nu_pts - nu[t]) <= cut)[0]
            if inside.size == 0:
                assert not keep[t]
                continue
            assert keep[t]
            # the index formulas and the distance test agree except exactly at a rounding tie
            assert abs(ilo[t] - inside[0]) <= 1 and abs(ihi[t] - inside[-1]) <= 1
            for i in (ilo[t], ihi[t]):
                assert abs(nu_pts[i] - nu[t]) <= cut * (1 + 1e-12)
            if ilo[t] > 0:
                assert abs(nu_pts[ilo[t] - 1] - nu[t]) > cut * (1 - 1e-12)
            if ihi[t] < n - 1:
                assert abs(nu_pts[ihi[t] + 1] - nu[t]) > cut * (1 - 1e-12)


@pytest.mark.parametrize("kind", ["voigt", "gauss_doppler", "lorentz", "pv_olivero"])
def test_sigma_equals_the_wavenumber_path_at_each_point(kind):
    E, g, up, lo, A, gr, ne = _tiny()
    lam0, dlam, n, cut = 1200.0, 0.05, 4000, 10.0
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind=kind, T=700.0, P=0.5, nu_min=lam0, dnu=dlam, n_grid=n,
                   cut=cut, wl_unit=NM)
    assert r["keep"].any()
    rng = np.random.default_rng(2)
    pts = np.concatenate([rng.integers(0, n, 60), [0, n - 1]])
    for i in pts:
        nu_i = NM / (lam0 + i * dlam)
        one = oracle.run(E, g, None, up, lo, A, gr, ne, kind=kind, T=700.0, P=0.5, nu_min=nu_i, dnu=1.0, n_grid=1,
                         cut=cut)
        assert r["sigma"][i] == pytest.approx(one["sigma"][0], rel=1e-11, abs=1e-300)


def test_nm_and_um_grids_agree():
    E, g, up, lo, A, gr, ne = _tiny(seed=5)
    a = oracle.run(E, g, None, up, lo, A, gr, ne, kind="voigt", T=900.0, P=1.0, nu_min=1500.0, dnu=0.04, n_grid=5000,
                   cut=8.0, wl_unit=NM)
    b = oracle.run(E, g, None, up, lo, A, gr, ne, kind="voigt", T=900.0, P=1.0, nu_min=1.5, dnu=0.00004,
                   n_grid=5000, cut=8.0, wl_unit=UM)
    assert np.array_equal(a["keep"], b["keep"])
    assert np.max(np.abs(a["sigma"] - b["sigma"])) <= 1e-9 * np.abs(a["sigma"]).max()


def test_isolated_line_peaks_at_its_wavelength_and_order_keeps_windows_monotone():
    E = np.array([0.0, 5000.0, 5000.0, 4000.0, 6000.0]); g = np.ones(5, np.int32)
    up = np.array([1, 3, 2, 4], np.int32); lo = np.zeros(4, np.int32); A = np.ones(4)
    gr = np.full(4, 0.01, np.float32); ne = np.full(4, 0.5, np.float32)
    lam0, dlam, n = 1600.0, 0.001, 1000001   # 1600 .. 2600 nm
    r = oracle.run(E, g, None, up, lo, A, gr, ne, kind="voigt", T=300.0, P=0.1, nu_min=lam0, dnu=dlam, n_grid=n,
                   cut=2.0, wl_unit=NM)
    # the line at 5000 cm^-1 sits at 2000 nm; its peak is at the nearest point
    i_line = int(round((NM / 5000.0 - lam0) / dlam))
    seg = r["sigma"][i_line - 2000:i_line + 2000]
    assert int(np.argmax(seg)) + i_line - 2000 == i_line
    # descending nu (6000, 5000, 5000, 4000 cm^-1), the equal pair by transition index
    assert list(r["perm"]) == [3, 0, 2, 1]
    ilo, ihi = r["ilo"][r["perm"]], r["ihi"][r["perm"]]
    assert np.all(np.diff(ilo) >= 0) and np.all(np.diff(ihi) >= 0)
