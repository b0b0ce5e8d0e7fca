"""FP64 CPU oracle (test infrastructure only).

Plain, slow, obviously-correct double-precision implementation of the
line-list -> intensity -> cross-section path of PyExoCross 2.0 (Secs. 2.4.2,
2.4.3, 3.1, 3.2) and of its adjoint.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg use it; the product path never imports it.  It
shares no code with the CUDA library (see oracle.c for the equations and the
readings taken where the text is silent).

Every function is pinned in tests/test_oracle.py against closed forms,
invariants, SciPy's independent Faddeeva implementation and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

KIND = {"gauss_doppler": 0, "gauss_hwhm": 1, "lorentz": 2, "voigt": 3,
        "binned_gauss_doppler": 4, "binned_gauss_hwhm": 5, "binned_lorentz": 6, "binned_voigt": 7,
        "pv_thompson": 8, "pv_olivero": 9, "pv_liulin": 10}
STATUS = {0: "ok", 1: "bad argument", 2: "state id out of range", 3: "non-finite input",
          4: "Boltzmann exponent overflow"}


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.orc_c2.restype = dbl
        L.orc_set_threads.argtypes = [cint]
        L.orc_faddeeva.argtypes = [i64, P, P, P, P]
        L.orc_profile.argtypes = [cint, i64, P, dbl, dbl, P, P, P]
        L.orc_partition.argtypes = [P, P, P, i64, dbl, dbl, P]
        L.orc_profile_binned.argtypes = [cint, i64, P, dbl, dbl, dbl, P]
        L.orc_pv_params.argtypes = [cint, i64, P, P, P, P, P]
        L.orc_line_intensities.argtypes = [P, P, P, i64, P, P, P, cint, i64, dbl, dbl, dbl,
                                           dbl, dbl, i64, dbl, dbl, dbl, P, P, P, P, P]
        L.orc_partition_density.argtypes = [P, P, P, P, i64, dbl, P]
        L.orc_intensities.argtypes = [cint, P, P, P, P, i64, P, P, P, cint, i64, dbl, dbl, dbl,
                                      dbl, dbl, i64, dbl, dbl, dbl, P, P, P, P, P]
        L.orc_cooling_function.argtypes = [P, P, P, P, i64, P, P, P, cint, i64, dbl, dbl, dbl, P]
        L.orc_list_exponent.argtypes = [P, P, i64]
        L.orc_list_exponent.restype = ctypes.c_int32
        L.orc_scale_intensities.argtypes = [P, P, i64, ctypes.c_int32, P]
        L.orc_sorted_order.argtypes = [P, P, i64, dbl, P]
        L.orc_sorted_order.restype = i64
        L.orc_segment_ranges.argtypes = [P, P, i64, i64, i64, P, P]
        L.orc_widths.argtypes = [cint, P, P, P, i64, dbl, dbl, dbl, dbl, dbl, P, P]
        L.orc_cross_section.argtypes = [cint, P, P, P, P, P, P, P, i64, dbl, dbl, i64, dbl, P]
        L.orc_cross_section_window.argtypes = [cint, P, P, P, P, P, P, P, i64, dbl, dbl, i64, i64, dbl, P]
        L.orc_cross_section_grad.argtypes = [cint, P, P, P, P, P, cint, P, P, P, P, P, P, P, P, i64,
                                             dbl, dbl, dbl, dbl, P, dbl, dbl, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}: {STATUS.get(code, '?')}")
        self.code = code


def _chk(code):
    if code != 0:
        raise OracleError(code)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's parallel loops use."""
    _load().orc_set_threads(int(n))


def c2() -> float:
    """Second radiation constant hc/k_B in cm K (CODATA 2018 exact values)."""
    return _load().orc_c2()


def faddeeva(x, y):
    """w(x + iy) for y >= 0, as complex128."""
    x = _c(np.atleast_1d(x), np.float64); y = _c(np.broadcast_to(y, x.shape), np.float64)
    re = np.empty_like(x); im = np.empty_like(x)
    _load().orc_faddeeva(x.size, _p(x), _p(y), _p(re), _p(im))
    return re + 1j * im


def profile(kind: str, x, alpha: float, gamma: float = 0.0, derivs: bool = False):
    """f(x) (and df/dalpha, df/dgamma) for one line with HWHMs alpha, gamma."""
    x = _c(np.atleast_1d(x), np.float64)
    f = np.empty_like(x); fa = np.empty_like(x); fg = np.empty_like(x)
    _load().orc_profile(KIND[kind], x.size, _p(x), alpha, gamma, _p(f), _p(fa), _p(fg))
    return (f, fa, fg) if derivs else f


def profile_binned(kind: str, x, dnu: float, alpha: float, gamma: float = 0.0):
    """Average of the profile `kind` ("gauss_*", "lorentz", "voigt" or their "binned_" names) over
    the bins [x - dnu/2, x + dnu/2]."""
    x = _c(np.atleast_1d(x), np.float64)
    f = np.empty_like(x)
    _load().orc_profile_binned(KIND[kind.replace("binned_", "")], x.size, _p(x), dnu, alpha, gamma, _p(f))
    return f


def pv_params(kind: str, alpha, gamma):
    """(G, w_L, w_G) of a pseudo-Voigt kind: the common full width and the weights of its
    Lorentzian and Gaussian, from Doppler and Lorentz HWHMs (reading R20 in oracle.c)."""
    a = _c(np.atleast_1d(alpha), np.float64); g = _c(np.broadcast_to(gamma, a.shape), np.float64)
    G = np.empty_like(a); wl = np.empty_like(a); wg = np.empty_like(a)
    _load().orc_pv_params(KIND[kind], a.size, _p(a), _p(g), _p(G), _p(wl), _p(wg))
    return G, wl, wg


def partition(E, g, E_vib=None, T=296.0, T_vib=0.0):
    """(Q, dQ/dT or dQ/dT_rot, dQ/dT_vib): Eq. (pf) or Eq. (Q nlte 2T)."""
    E = _c(E, np.float64); g = _c(g, np.int32); Ev = _c(E_vib, np.float64)
    out = np.zeros(3)
    _chk(_load().orc_partition(_p(E), _p(g), _p(Ev), E.size, T, T_vib, _p(out)))
    return out


def line_intensities(E, g, E_vib, upper, lower, A, T, T_vib, Q, nu_min, dnu, n_grid, cut, threshold=0.0,
                     wl_unit=0.0):
    """Per-transition nu, I (cm/molecule, 0 where dropped), keep, ilo, ihi.  wl_unit > 0 makes the
    grid (nu_min, dnu) a wavelength grid in that unit (1e7: nm, 1e4: um; reading R21)."""
    E = _c(E, np.float64); g = _c(g, np.int32); Ev = _c(E_vib, np.float64)
    up = _c(upper, np.int32); lo = _c(lower, np.int32)
    A_f32 = A.dtype == np.float32
    A = _c(A, np.float32 if A_f32 else np.float64)
    n = up.size
    nu = np.empty(n); I = np.empty(n); keep = np.empty(n, np.uint8)
    ilo = np.empty(n, np.int64); ihi = np.empty(n, np.int64)
    _chk(_load().orc_line_intensities(_p(E), _p(g), _p(Ev), E.size, _p(up), _p(lo), _p(A), int(A_f32), n,
                                      T, T_vib, Q, nu_min, dnu, n_grid, cut, threshold, wl_unit,
                                      _p(nu), _p(I), _p(keep), _p(ilo), _p(ihi)))
    return nu, I, keep, ilo, ihi


def partition_density(E, g, E_vib, n_vib, T_rot):
    """(Q, dQ/dT_rot) with vibronic densities: Eq. (Q nlte Nvib)."""
    E = _c(E, np.float64); g = _c(g, np.int32); Ev = _c(E_vib, np.float64); nv = _c(n_vib, np.float64)
    out = np.zeros(2)
    _chk(_load().orc_partition_density(_p(E), _p(g), _p(Ev), _p(nv), E.size, T_rot, _p(out)))
    return out


def intensities(E, g, E_vib, upper, lower, A, T, T_vib, Q, nu_min, dnu, n_grid, cut, threshold=0.0,
                emission=False, n_vib=None, wl_unit=0.0):
    """Per-transition nu, value (absorption cm/molecule or emission erg/s/sr/molecule), keep, ilo, ihi
    for the LTE, two-temperature (T_vib > 0) or vibronic-density (n_vib given) populations."""
    E = _c(E, np.float64); g = _c(g, np.int32); Ev = _c(E_vib, np.float64); nv = _c(n_vib, np.float64)
    up = _c(upper, np.int32); lo = _c(lower, np.int32)
    A_f32 = A.dtype == np.float32
    A = _c(A, np.float32 if A_f32 else np.float64)
    n = up.size
    nu = np.empty(n); I = np.empty(n); keep = np.empty(n, np.uint8)
    ilo = np.empty(n, np.int64); ihi = np.empty(n, np.int64)
    _chk(_load().orc_intensities(int(bool(emission)), _p(E), _p(g), _p(Ev), _p(nv), E.size, _p(up), _p(lo), _p(A),
                                 int(A_f32), n, T, T_vib, Q, nu_min, dnu, n_grid, cut, threshold, wl_unit,
                                 _p(nu), _p(I), _p(keep), _p(ilo), _p(ihi)))
    return nu, I, keep, ilo, ihi


def cooling_function(E, g, E_vib, upper, lower, A, T, T_vib, Q, n_vib=None) -> float:
    """W(T) in erg/s/sr/molecule: Eq. (cf), and its non-LTE forms (sum of emission intensities)."""
    E = _c(E, np.float64); g = _c(g, np.int32); Ev = _c(E_vib, np.float64); nv = _c(n_vib, np.float64)
    up = _c(upper, np.int32); lo = _c(lower, np.int32)
    A_f32 = A.dtype == np.float32
    A = _c(A, np.float32 if A_f32 else np.float64)
    W = np.zeros(1)
    _chk(_load().orc_cooling_function(_p(E), _p(g), _p(Ev), _p(nv), E.size, _p(up), _p(lo), _p(A), int(A_f32),
                                      up.size, T, T_vib, Q, _p(W)))
    return float(W[0])


def list_exponent(I, keep) -> int:
    I = _c(I, np.float64); keep = _c(keep, np.uint8)
    return int(_load().orc_list_exponent(_p(I), _p(keep), I.size))


def scale_intensities(I, keep, k):
    I = _c(I, np.float64); keep = _c(keep, np.uint8)
    out = np.empty(I.size, np.float32)
    _load().orc_scale_intensities(_p(I), _p(keep), I.size, int(k), _p(out))
    return out


def sorted_order(nu, keep, wl_unit=0.0):
    """Kept transition indices in ascending (nu bits, index) order (descending nu bits on a
    wavelength grid)."""
    nu = _c(nu, np.float64); keep = _c(keep, np.uint8)
    perm = np.empty(nu.size, np.int64)
    m = _load().orc_sorted_order(_p(nu), _p(keep), nu.size, wl_unit, _p(perm))
    return perm[:m].copy()


def segment_ranges(ilo_sorted, ihi_sorted, n_grid, S):
    a = _c(ilo_sorted, np.int64); b = _c(ihi_sorted, np.int64)
    nseg = (n_grid + S - 1) // S
    first = np.empty(nseg, np.int64); last = np.empty(nseg, np.int64)
    _load().orc_segment_ranges(_p(a), _p(b), a.size, n_grid, S, _p(first), _p(last))
    return first, last


def widths(kind, nu, gamma_ref, n_T, T, P, mass_da=18.0, hwhm=0.0, T_ref=296.0):
    nu = _c(nu, np.float64)
    gr = _c(gamma_ref if gamma_ref is not None else np.zeros(nu.size), np.float32)
    ne = _c(n_T if n_T is not None else np.zeros(nu.size), np.float32)
    a = np.empty(nu.size); gm = np.empty(nu.size)
    _load().orc_widths(KIND[kind], _p(nu), _p(gr), _p(ne), nu.size, T, P, mass_da, hwhm, T_ref, _p(a), _p(gm))
    return a, gm


def cross_section(kind, nu, I, alpha, gamma, keep, ilo, ihi, nu_min, dnu, n_grid, wl_unit=0.0):
    """sigma on the grid (cm^2/molecule), Eq. (xsec)."""
    nu = _c(np.where(keep.astype(bool), nu, 0.0), np.float64)
    I = _c(I, np.float64); alpha = _c(alpha, np.float64); gamma = _c(gamma, np.float64)
    keep = _c(keep, np.uint8); ilo = _c(ilo, np.int64); ihi = _c(ihi, np.int64)
    sig = np.empty(n_grid)
    _chk(_load().orc_cross_section(KIND[kind], _p(nu), _p(I), _p(alpha), _p(gamma), _p(keep), _p(ilo), _p(ihi),
                                   nu.size, nu_min, dnu, n_grid, wl_unit, _p(sig)))
    return sig


def cross_section_window(kind, nu, I, alpha, gamma, keep, ilo, ihi, nu_min, dnu, i0, m, wl_unit=0.0):
    """sigma at grid indices i0 .. i0+m-1 only (same grid points as the full grid)."""
    nu = _c(np.where(keep.astype(bool), nu, 0.0), np.float64)
    I = _c(I, np.float64); alpha = _c(alpha, np.float64); gamma = _c(gamma, np.float64)
    keep = _c(keep, np.uint8); ilo = _c(ilo, np.int64); ihi = _c(ihi, np.int64)
    sig = np.empty(m)
    _chk(_load().orc_cross_section_window(KIND[kind], _p(nu), _p(I), _p(alpha), _p(gamma), _p(keep), _p(ilo),
                                          _p(ihi), nu.size, nu_min, dnu, i0, m, wl_unit, _p(sig)))
    return sig


def cross_section_grad(kind, E, E_vib, upper, lower, A, nu, I, alpha, gamma, n_T, keep, ilo, ihi,
                       T, T_vib, P, Qd, nu_min, dnu, w, T_ref=296.0):
    """Adjoint of L = sum_i w_i sigma_i.  Returns dict of FP64 gradients and scales."""
    E = _c(E, np.float64); Ev = _c(E_vib, np.float64)
    up = _c(upper, np.int32); lo = _c(lower, np.int32)
    A_f32 = A.dtype == np.float32
    A = _c(A, np.float32 if A_f32 else np.float64)
    nu = _c(np.where(keep.astype(bool), nu, 1.0), np.float64)
    I = _c(I, np.float64); alpha = _c(alpha, np.float64); gamma = _c(gamma, np.float64)
    ne = _c(n_T if n_T is not None else np.zeros(nu.size), np.float32)
    keep = _c(keep, np.uint8); ilo = _c(ilo, np.int64); ihi = _c(ihi, np.int64)
    Qd = _c(Qd, np.float64); w = _c(w, np.float64)
    n = nu.size
    dA = np.empty(n); dg = np.empty(n); G = np.empty((n, 3)); Gabs = np.empty((n, 3)); scal = np.empty(6)
    _chk(_load().orc_cross_section_grad(KIND[kind], _p(E), _p(Ev), _p(up), _p(lo), _p(A), int(A_f32),
                                        _p(nu), _p(I), _p(alpha), _p(gamma), _p(ne), _p(keep), _p(ilo), _p(ihi),
                                        n, T, T_vib, P, T_ref, _p(Qd), nu_min, dnu, _p(w),
                                        _p(dA), _p(dg), _p(G), _p(Gabs), _p(scal)))
    return {"dA": dA, "dgamma_ref": dg, "G": G, "Gabs": Gabs,
            "dT": scal[0], "dTvib": scal[1], "dP": scal[2],
            "dT_abs": scal[3], "dTvib_abs": scal[4], "dP_abs": scal[5]}


def run(E, g, E_vib, upper, lower, A, gamma_ref, n_T, *, kind, T, T_vib=0.0, P=1.0, mass_da=18.0,
        hwhm=0.0, nu_min, dnu, n_grid, cut, threshold=0.0, T_ref=296.0, with_sigma=True,
        emission=False, n_vib=None, wl_unit=0.0):
    """Whole forward path: Q, per-line quantities, exponent, sort order, sigma (absorption or
    emission; LTE, two-temperature or vibronic-density populations)."""
    if n_vib is not None:
        Qd = np.append(partition_density(E, g, E_vib, n_vib, T), 0.0)
    else:
        Qd = partition(E, g, E_vib if T_vib > 0 else None, T, T_vib)
    if emission or n_vib is not None:
        nu, I, keep, ilo, ihi = intensities(E, g, E_vib, upper, lower, A, T, T_vib, Qd[0], nu_min, dnu, n_grid,
                                            cut, threshold, emission=emission, n_vib=n_vib, wl_unit=wl_unit)
    else:
        nu, I, keep, ilo, ihi = line_intensities(E, g, E_vib, upper, lower, A, T, T_vib, Qd[0],
                                                 nu_min, dnu, n_grid, cut, threshold, wl_unit=wl_unit)
    k = list_exponent(I, keep)
    I_s = scale_intensities(I, keep, k)
    perm = sorted_order(nu, keep, wl_unit)
    nu_w = np.where(keep.astype(bool), nu, 1.0)
    alpha, gamma = widths(kind, nu_w, gamma_ref, n_T, T, P, mass_da, hwhm, T_ref)
    out = {"Q": Qd, "nu": nu, "I": I, "keep": keep, "ilo": ilo, "ihi": ihi, "k": k, "I_s": I_s,
           "perm": perm, "alpha": alpha, "gamma": gamma,
           "evals": int(np.sum((ihi - ilo + 1)[keep.astype(bool)]))}
    if with_sigma:
        out["sigma"] = cross_section(kind, nu, I, alpha, gamma, keep, ilo, ihi, nu_min, dnu, n_grid, wl_unit)
    return out
