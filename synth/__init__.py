"""Seeded synthetic line lists for the cross-section workloads.

Inputs only: this package computes no partition function, intensity, profile or
cross section.  Both the FP64 oracle and the CUDA path consume the arrays it
returns; neither imports the other.  The C generator (synth.c) is built on first
use with gcc and OpenMP; its output does not depend on the thread count.

Workloads (sizes follow the line-list shapes of Sec. 2.3 and the LTE / non-LTE
formulation of Sec. 3):
  doppler_1e5  5,000 diatomic states, 1e5 transitions, Doppler profile
  voigt_1e7    1e6 diatomic states, 1e7 transitions, Voigt profile
  voigt_1e9    5e7 polyatomic states, 1e9 transitions (1e8 chunks), Voigt
  table_1e8    voigt_1e7's generator at 1e8 transitions, 20 T x 10 P conditions
  nlte_1e7     voigt_1e7's list with T_vib = 2500 K, T_rot = 1200 K
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _synth.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u64, dbl, ptr = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.synth_states_diatomic.argtypes = [i64, i64, ctypes.c_int, ptr, ptr, ptr]
        lib.synth_transitions_diatomic.argtypes = [u64, i64, i64, i64, i64, dbl, dbl, ptr, ptr, ptr, ptr]
        lib.synth_states_polyatomic.argtypes = [u64, i64, i64, ptr, ptr, ptr]
        lib.synth_transitions_polyatomic.argtypes = [u64, i64, i64, i64, dbl, dbl, ptr, ptr, ptr, ptr]
        lib.synth_uniform_f32.argtypes = [u64, ctypes.c_int, i64, i64, dbl, dbl, ptr]
        lib.synth_normal_f32.argtypes = [u64, i64, ptr]
        lib.synth_draw64.argtypes = [u64, u64, u64]
        lib.synth_draw64.restype = u64
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


ST_GAMMA, ST_NEXP, ST_VIBDENS = 4, 5, 9


@dataclass
class Workload:
    """One synthetic workload: level scheme, list size, conditions, grid, profile."""
    name: str
    seed: int
    scheme: str                  # "diatomic" | "polyatomic"
    n_states: int
    n_trans: int
    nv: int = 0
    nJ: int = 0
    logA: tuple = (-6.0, 2.0)
    A_f32: bool = False
    T: float = 296.0
    T_vib: float = 0.0           # > 0: two-temperature non-LTE, T is T_rot
    P: float = 1.0
    mass_da: float = 18.0
    profile: str = "voigt"       # gauss_doppler | gauss_hwhm | lorentz | voigt
    hwhm: float = 0.0
    nu_min: float = 0.0
    dnu: float = 0.01
    n_grid: int = 2_000_001
    cutoff: float = 25.0
    threshold: float = 0.0
    chunk: int = 0               # > 0: transitions streamed in chunks of this size
    gamma_range: tuple = (0.03, 0.10)
    n_range: tuple = (0.4, 0.8)
    conditions: list = field(default_factory=list)  # batched (T, P) pairs

    def states(self, literal: bool = False, id0: int = 0, n: int | None = None):
        """(E[f64], g[i32], E_vib[f64]) for state ids id0 .. id0+n-1."""
        lib = _load()
        if self.scheme == "diatomic":
            E = np.empty(self.nv * self.nJ)
            g = np.empty(self.nv * self.nJ, np.int32)
            Ev = np.empty(self.nv * self.nJ)
            lib.synth_states_diatomic(self.nv, self.nJ, int(literal), _p(E), _p(g), _p(Ev))
            n = self.n_states - id0 if n is None else n
            return E[id0:id0 + n].copy(), g[id0:id0 + n].copy(), Ev[id0:id0 + n].copy()
        n = self.n_states - id0 if n is None else n
        E = np.empty(n); g = np.empty(n, np.int32); Ev = np.empty(n)
        lib.synth_states_polyatomic(self.seed, id0, n, _p(E), _p(g), _p(Ev))
        return E, g, Ev

    def transitions(self, t0: int = 0, n: int | None = None, out=None):
        """(upper[i32], lower[i32], A[f64 or f32]) for transitions t0 .. t0+n-1.

        `out` may supply preallocated (upper, lower, A) arrays (e.g. pinned memory)."""
        lib = _load()
        n = self.n_trans - t0 if n is None else n
        if out is None:
            up = np.empty(n, np.int32); lo = np.empty(n, np.int32)
            A = np.empty(n, np.float32 if self.A_f32 else np.float64)
        else:
            up, lo, A = out
        a64 = None if self.A_f32 else A
        a32 = A if self.A_f32 else None
        if self.scheme == "diatomic":
            lib.synth_transitions_diatomic(self.seed, self.nv, self.nJ, t0, n, self.logA[0], self.logA[1],
                                           _p(up), _p(lo), _p(a64), _p(a32))
        else:
            lib.synth_transitions_polyatomic(self.seed, self.n_states, t0, n, self.logA[0], self.logA[1],
                                             _p(up), _p(lo), _p(a64), _p(a32))
        return up, lo, A

    def broadening(self, t0: int = 0, n: int | None = None):
        """(gamma_ref[f32] in cm^-1/bar, n_T[f32]) per transition."""
        lib = _load()
        n = self.n_trans - t0 if n is None else n
        gr = np.empty(n, np.float32); ne = np.empty(n, np.float32)
        lib.synth_uniform_f32(self.seed, ST_GAMMA, t0, n, self.gamma_range[0], self.gamma_range[1], _p(gr))
        lib.synth_uniform_f32(self.seed, ST_NEXP, t0, n, self.n_range[0], self.n_range[1], _p(ne))
        return gr, ne

    def vib_densities(self) -> np.ndarray:
        """Per-state custom vibronic densities n_vib[f64] for a diatomic level scheme: one
        seeded, non-thermal weight per vibrational manifold, (0.5 + U) exp(-v / 2.5), normalised
        to sum 1 over the manifolds; every rotational state of manifold v carries its weight."""
        if self.scheme != "diatomic":
            raise ValueError("vibronic densities are generated for diatomic level schemes")
        u = np.empty(self.nv, np.float32)
        _load().synth_uniform_f32(self.seed, ST_VIBDENS, 0, self.nv, 0.0, 1.0, _p(u))
        v = np.arange(self.nv)
        w = (0.5 + u.astype(np.float64)) * np.exp(-v / 2.5)
        w /= w.sum()
        return np.repeat(w, self.nJ)[: self.n_states].copy()

    def weights(self, n: int | None = None, seed_offset: int = 7):
        """Seeded N(0,1) loss weights w(nu) on the grid."""
        lib = _load()
        n = self.n_grid if n is None else n
        w = np.empty(n, np.float32)
        lib.synth_normal_f32(self.seed + seed_offset, n, _p(w))
        return w

    def grid(self):
        return self.nu_min + np.arange(self.n_grid) * self.dnu

    def scaled(self, **kw) -> "Workload":
        """A copy with some fields replaced (used for small parity cases)."""
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


BASE_SEED = 20260917


def _table_conditions():
    Ts = np.geomspace(200.0, 3000.0, 20)
    Ps = np.geomspace(1e-5, 100.0, 10)
    return [(float(t), float(p)) for t in Ts for p in Ps]


WORKLOADS = {
    "doppler_1e5": Workload("doppler_1e5", BASE_SEED + 1, "diatomic", 5000, 100_000, nv=5, nJ=1000,
                            logA=(-6.0, 2.0), T=1000.0, profile="gauss_doppler",
                            nu_min=0.0, dnu=0.1, n_grid=100_001, cutoff=25.0),
    "voigt_1e7": Workload("voigt_1e7", BASE_SEED + 2, "diatomic", 1_000_000, 10_000_000, nv=10, nJ=100_000,
                          logA=(-6.0, 2.0), T=1500.0, P=1.0, profile="voigt",
                          nu_min=0.0, dnu=0.01, n_grid=2_000_001, cutoff=25.0),
    "voigt_1e9": Workload("voigt_1e9", BASE_SEED + 3, "polyatomic", 50_000_000, 1_000_000_000,
                          logA=(-8.0, 3.0), A_f32=True, T=2000.0, P=0.1, profile="voigt",
                          nu_min=0.0, dnu=0.01, n_grid=3_000_001, cutoff=25.0, threshold=1e-30,
                          chunk=100_000_000),
    "table_1e8": Workload("table_1e8", BASE_SEED + 4, "diatomic", 1_000_000, 100_000_000, nv=10, nJ=100_000,
                          logA=(-6.0, 2.0), T=1500.0, P=1.0, profile="voigt",
                          nu_min=0.0, dnu=0.01, n_grid=2_000_001, cutoff=25.0,
                          conditions=_table_conditions()),
    "nlte_1e7": Workload("nlte_1e7", BASE_SEED + 5, "diatomic", 1_000_000, 10_000_000, nv=10, nJ=100_000,
                         logA=(-6.0, 2.0), T=1200.0, T_vib=2500.0, P=1.0, profile="voigt",
                         nu_min=0.0, dnu=0.01, n_grid=2_000_001, cutoff=25.0),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
