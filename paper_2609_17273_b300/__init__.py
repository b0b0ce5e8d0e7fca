"""Python binding of the pxc C ABI (include/pxc.h): line list -> intensities -> cross sections.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libpxc.so (built in-tree for sm_103a by build.py).  PyTorch supplies
device memory and streams.  There is no CPU fallback: importing the binding
without the built library, or calling it without a CUDA device, raises.

The function names are those of the ABI; see include/pxc.h for the contract of
each call (units, layouts, ownership, error behaviour).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpxc.so")

PXC_GAUSS_DOPPLER, PXC_GAUSS_HWHM, PXC_LORENTZ, PXC_VOIGT = 0, 1, 2, 3
PROFILES = {"gauss_doppler": 0, "gauss_hwhm": 1, "lorentz": 2, "voigt": 3,
            "binned_gauss_doppler": 4, "binned_gauss_hwhm": 5, "binned_lorentz": 6, "binned_voigt": 7,
            "pv_thompson": 8, "pv_olivero": 9, "pv_liulin": 10}
# Kinds whose widths include the pressure (Lorentz) width, so need gamma_ref and n_T.
BROADENED = ("lorentz", "voigt", "binned_lorentz", "binned_voigt", "pv_thompson", "pv_olivero", "pv_liulin")
# Wavelength units of a grid (nu = unit / lambda): pass as the grid's fourth element.
WL_NM, WL_UM = 1e7, 1e4
PXC_EXP_EMPTY = -2147483648
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_ID_RANGE", 3: "ERR_NONFINITE", 4: "ERR_OVERFLOW", 5: "ERR_TIMEOUT",
          6: "ERR_CUDA", 7: "ERR_CAPACITY"}

c_i32, c_i64, c_dbl, c_ptr = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class pxc_states(ctypes.Structure):
    _fields_ = [("E", c_ptr), ("g", c_ptr), ("E_vib", c_ptr), ("n", c_i64), ("n_vib", c_ptr)]


class pxc_transitions(ctypes.Structure):
    _fields_ = [("upper", c_ptr), ("lower", c_ptr), ("A", c_ptr), ("A_is_f32", c_i32), ("n", c_i64)]


class pxc_condition(ctypes.Structure):
    _fields_ = [("T", c_dbl), ("T_vib", c_dbl), ("P", c_dbl)]


class pxc_grid(ctypes.Structure):
    """(nu_min, dnu, n[, wl_unit]): wavenumbers, or wavelengths in the unit wl_unit (1e7 nm, 1e4 um)."""
    _fields_ = [("nu_min", c_dbl), ("dnu", c_dbl), ("n", c_i64), ("wl_unit", c_dbl)]


class pxc_profile_args(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("cutoff", c_dbl), ("mass_da", c_dbl), ("hwhm", c_dbl),
                ("gamma_ref", c_ptr), ("n_T", c_ptr), ("T_ref", c_dbl)]


class pxc_capacity(ctypes.Structure):
    _fields_ = [("max_states", c_i64), ("max_lines", c_i64), ("max_grid", c_i64),
                ("max_conditions", c_i32), ("max_temperatures", c_i32)]


class pxc_stats(ctypes.Structure):
    _fields_ = [("n_kept", c_i64), ("n_nonzero", c_i64), ("evals_window", c_i64), ("evals_nonzero", c_i64),
                ("segment_points", c_i32), ("n_segments", c_i32), ("I_exp", c_i32), ("tile", c_i32)]


class PxcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# Names the header declares; the CPU tests check that the library exports each.
ABI_FUNCTIONS = [
    "pxc_workspace_query", "pxc_workspace_create", "pxc_workspace_destroy", "pxc_sync_status", "pxc_last_error",
    "pxc_set_accumulate", "pxc_partition_function", "pxc_line_intensities", "pxc_cross_section",
    "pxc_cross_section_backward", "pxc_get_stats", "pxc_get_binning", "pxc_stream_buffer_bytes",
    "pxc_cross_section_streamed", "pxc_kernel_launches", "pxc_set_timing", "pxc_get_timing",
    "pxc_partition_function_noalloc", "pxc_set_tile", "pxc_get_tile", "pxc_autotune",
    "pxc_set_emission", "pxc_cooling_function", "pxc_set_wait_limit", "pxc_pipe_rates_buffer_bytes",
    "pxc_pipe_rates", "pxc_set_graphs", "pxc_graph_stats", "pxc_set_reuse_forward",
]

# Profile-kernel tile configurations (segment width in grid points), as compiled into the library.
NUM_TILES = 4
TILE_SEGMENT_POINTS = (128, 256, 1024, 2048)
BATCHED_DEFAULT_TILE = 0


def load(path: str | None = None):
    """Load libpxc.so (or the build named by PXC_LIBRARY); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PXC_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libpxc.so not built ({path}); run paper_2609_17273_b300/build.py")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.pxc_last_error.restype = ctypes.c_char_p
    L.pxc_kernel_launches.restype = c_i64
    L.pxc_workspace_query.argtypes = [P(pxc_capacity), P(ctypes.c_size_t)]
    L.pxc_workspace_create.argtypes = [P(pxc_capacity), c_ptr, ctypes.c_size_t, P(c_ptr)]
    L.pxc_workspace_destroy.argtypes = [c_ptr]
    L.pxc_sync_status.argtypes = [c_ptr, c_ptr]
    L.pxc_set_accumulate.argtypes = [c_ptr, ctypes.c_int]
    L.pxc_partition_function.argtypes = [c_ptr, P(pxc_states), P(pxc_condition), c_i32, c_ptr, c_ptr, c_ptr]
    L.pxc_line_intensities.argtypes = [c_ptr, P(pxc_states), P(pxc_transitions), P(pxc_condition), P(pxc_grid),
                                       c_dbl, c_dbl, c_ptr, c_ptr, c_ptr, c_ptr, c_ptr]
    L.pxc_cross_section.argtypes = [c_ptr, P(pxc_states), P(pxc_transitions), P(pxc_condition), c_i32,
                                    P(pxc_grid), P(pxc_profile_args), c_dbl, c_ptr, c_ptr, c_ptr]
    L.pxc_cross_section_backward.argtypes = [c_ptr, P(pxc_states), P(pxc_transitions), P(pxc_condition), c_i32,
                                             P(pxc_grid), P(pxc_profile_args), c_dbl, c_ptr, c_ptr, c_ptr, c_ptr,
                                             c_ptr, c_ptr, c_ptr]
    L.pxc_get_stats.argtypes = [c_ptr, c_ptr, P(pxc_stats)]
    L.pxc_get_binning.argtypes = [c_ptr, c_ptr, c_ptr, c_ptr, c_ptr]
    L.pxc_partition_function_noalloc.argtypes = [P(pxc_states), P(pxc_condition), c_i32, c_ptr, c_ptr, c_ptr,
                                                 c_ptr]
    L.pxc_set_timing.argtypes = [c_ptr, ctypes.c_int]
    L.pxc_get_timing.argtypes = [c_ptr, c_ptr, c_ptr, c_ptr]
    L.pxc_set_emission.argtypes = [c_ptr, ctypes.c_int]
    L.pxc_set_wait_limit.argtypes = [c_ptr, c_i64]
    L.pxc_set_graphs.argtypes = [c_ptr, ctypes.c_int]
    L.pxc_set_reuse_forward.argtypes = [c_ptr, ctypes.c_int32]
    L.pxc_graph_stats.argtypes = [c_ptr, P(c_i64), P(c_i64), P(c_i32)]
    L.pxc_cooling_function.argtypes = [c_ptr, P(pxc_states), P(pxc_transitions), P(pxc_condition), c_i32,
                                       c_ptr, c_ptr, c_ptr]
    L.pxc_set_tile.argtypes = [c_ptr, c_i32, c_i32, c_i32]
    L.pxc_get_tile.argtypes = [c_ptr, c_i32, c_i32, P(c_i32)]
    L.pxc_autotune.argtypes = [c_ptr, P(pxc_states), P(pxc_transitions), P(pxc_condition), c_i32, P(pxc_grid),
                               P(pxc_profile_args), c_dbl, c_ptr, c_ptr, c_i32, P(c_i32), c_ptr, c_ptr]
    L.pxc_stream_buffer_bytes.argtypes = [c_i64, c_i32, c_i32]
    L.pxc_stream_buffer_bytes.restype = ctypes.c_size_t
    L.pxc_cross_section_streamed.argtypes = [c_ptr, P(pxc_states), c_ptr, c_ptr, c_ptr, c_i32, c_ptr, c_ptr, c_i64,
                                             P(pxc_condition), P(pxc_grid), P(pxc_profile_args), c_dbl,
                                             c_ptr, c_ptr, ctypes.c_size_t, c_ptr, c_ptr, c_ptr]
    L.pxc_pipe_rates_buffer_bytes.argtypes = []
    L.pxc_pipe_rates_buffer_bytes.restype = ctypes.c_size_t
    L.pxc_pipe_rates.argtypes = [c_ptr, ctypes.c_size_t, c_ptr, c_ptr]
    for name in ABI_FUNCTIONS:
        fn = getattr(L, name)
        if name not in ("pxc_last_error", "pxc_stream_buffer_bytes", "pxc_kernel_launches",
                        "pxc_pipe_rates_buffer_bytes"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def kernel_launches() -> int:
    """Kernels launched by libpxc.so since load."""
    return int(load().pxc_kernel_launches())


def _check(code: int):
    if code != 0:
        raise PxcError(code, load().pxc_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name}: expected a contiguous CUDA tensor of {dtype}")
    return t


@dataclass
class States:
    """Device arrays of a .states table: E (float64), g (int32), E_vib (float64 or None), and
    optional custom vibronic densities n_vib (float64; selects the density populations)."""
    E: torch.Tensor
    g: torch.Tensor
    E_vib: torch.Tensor | None = None
    n_vib: torch.Tensor | None = None

    def c(self):
        _dev(self.E, torch.float64, "E"); _dev(self.g, torch.int32, "g"); _dev(self.E_vib, torch.float64, "E_vib")
        _dev(self.n_vib, torch.float64, "n_vib")
        return pxc_states(_ptr(self.E), _ptr(self.g), _ptr(self.E_vib), self.E.numel(), _ptr(self.n_vib))


@dataclass
class Transitions:
    """Device arrays of a .trans table: upper, lower (int32), A (float64 or float32)."""
    upper: torch.Tensor
    lower: torch.Tensor
    A: torch.Tensor

    def c(self):
        _dev(self.upper, torch.int32, "upper"); _dev(self.lower, torch.int32, "lower")
        if self.A.dtype not in (torch.float32, torch.float64) or not self.A.is_cuda:
            raise TypeError("A: expected a CUDA float32/float64 tensor")
        return pxc_transitions(_ptr(self.upper), _ptr(self.lower), _ptr(self.A),
                               int(self.A.dtype == torch.float32), self.upper.numel())


@dataclass
class Profile:
    """Line profile: kind in PROFILES, cut-off, mass (Da), fixed HWHM, per-line gamma_ref and n_T."""
    kind: str = "voigt"
    cutoff: float = 25.0
    mass_da: float = 18.0
    hwhm: float = 0.0
    gamma_ref: torch.Tensor | None = None
    n_T: torch.Tensor | None = None
    T_ref: float = 296.0

    def c(self):
        _dev(self.gamma_ref, torch.float32, "gamma_ref"); _dev(self.n_T, torch.float32, "n_T")
        return pxc_profile_args(PROFILES[self.kind], self.cutoff, self.mass_da, self.hwhm,
                                _ptr(self.gamma_ref), _ptr(self.n_T), self.T_ref)


def _conds(conds):
    if isinstance(conds, tuple) and len(conds) == 3 and not isinstance(conds[0], (tuple, list)):
        conds = [conds]
    arr = (pxc_condition * len(conds))()
    for i, (T, Tv, P) in enumerate(conds):
        arr[i] = pxc_condition(T, Tv, P)
    return arr, len(conds)


class Workspace:
    """Device scratch sized by pxc_workspace_query, owned here as a torch tensor."""

    def __init__(self, max_states: int, max_lines: int, max_grid: int, max_conditions: int = 1,
                 max_temperatures: int = 0, device="cuda"):
        L = load()
        self.cap = pxc_capacity(max_states, max_lines, max_grid, max_conditions, max_temperatures)
        nbytes = ctypes.c_size_t()
        _check(L.pxc_workspace_query(ctypes.byref(self.cap), ctypes.byref(nbytes)))
        self.nbytes = nbytes.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.buf.data_ptr()
        self.base = (base + 255) & ~255
        h = ctypes.c_void_p()
        _check(L.pxc_workspace_create(ctypes.byref(self.cap), ctypes.c_void_p(self.base), self.nbytes,
                                      ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().pxc_workspace_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """pxc_sync_status: synchronise and raise the latched device error, if any."""
        _check(load().pxc_sync_status(self.h, _stream(stream)))

    def stats(self, stream=None) -> dict:
        st = pxc_stats()
        _check(load().pxc_get_stats(self.h, _stream(stream), ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in pxc_stats._fields_}

    def binning(self, n_kept: int, n_segments: int, stream=None):
        perm = torch.empty(max(n_kept, 1), dtype=torch.int64, device="cuda")
        f = torch.empty(max(n_segments, 1), dtype=torch.int64, device="cuda")
        l = torch.empty(max(n_segments, 1), dtype=torch.int64, device="cuda")
        _check(load().pxc_get_binning(self.h, _ptr(perm), _ptr(f), _ptr(l), _stream(stream)))
        return perm[:n_kept], f[:n_segments], l[:n_segments]

    def set_timing(self, on: bool):
        _check(load().pxc_set_timing(self.h, int(on)))

    def timing(self, stream=None) -> dict:
        """Summed CUDA-event times (ms) and launch counts of the passes since the last read."""
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        _check(load().pxc_get_timing(self.h, _stream(stream), ms, cnt))
        names = ("intensity", "sort", "profile")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(names)}

    def set_accumulate(self, on: bool):
        _check(load().pxc_set_accumulate(self.h, int(on)))

    def set_wait_limit(self, cycles: int = 4_000_000_000):
        """Bound (clock cycles) of the profile kernel's waits for staged records; 0 forces timeouts."""
        _check(load().pxc_set_wait_limit(self.h, int(cycles)))

    def set_emission(self, on: bool):
        """Emission intensities / emission cross sections instead of absorption (workspace mode)."""
        _check(load().pxc_set_emission(self.h, int(on)))

    def set_graphs(self, on: bool):
        """Capture distinct pxc_cross_section calls into CUDA graphs and replay identical ones."""
        _check(load().pxc_set_graphs(self.h, int(on)))

    def set_reuse_forward(self, on: bool):
        """Let pxc_cross_section_backward reuse the line list of an identical preceding forward call
        (the caller guarantees the arrays are unchanged in between)."""
        _check(load().pxc_set_reuse_forward(self.h, int(on)))

    def graph_stats(self) -> dict:
        cap, rep, cached = c_i64(0), c_i64(0), c_i32(0)
        _check(load().pxc_graph_stats(self.h, ctypes.byref(cap), ctypes.byref(rep), ctypes.byref(cached)))
        return {"captures": int(cap.value), "replays": int(rep.value), "cached": int(cached.value)}

    def set_tile(self, kind: int, batched: bool, tile: int):
        """Profile-kernel tile for this kind and for single-condition (batched=False) or batched calls."""
        _check(load().pxc_set_tile(self.h, int(kind), int(bool(batched)), int(tile)))

    def get_tile(self, kind: int, batched: bool) -> int:
        t = c_i32(0)
        _check(load().pxc_get_tile(self.h, int(kind), int(bool(batched)), ctypes.byref(t)))
        return int(t.value)


def pxc_pipe_rates(stream=None) -> dict:
    """Measured FP32 FMA, MUFU rcp / ex2 and far-wing Voigt evaluation rates of the current device:
    per SM per clock cycle and per second (include/pxc.h, pxc_pipe_rates)."""
    L = load()
    nb = L.pxc_pipe_rates_buffer_bytes()
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * 8)()
    _check(L.pxc_pipe_rates(_ptr(buf), nb, out, _stream(stream)))
    names = ("fma", "rcp", "ex2", "voigt_far_eval")
    return {"per_sm_per_clk": {n: out[i] for i, n in enumerate(names)},
            "per_s": {n: out[4 + i] for i, n in enumerate(names)}}


def pxc_partition_function(ws: Workspace, states: States, conds, stream=None):
    """Q[n_c] (float64) and dQ[n_c, 2] on the device."""
    arr, n = _conds(conds)
    Q = torch.empty(n, dtype=torch.float64, device="cuda")
    dQ = torch.empty(n, 2, dtype=torch.float64, device="cuda")
    st = states.c()
    _check(load().pxc_partition_function(ws.h, ctypes.byref(st), arr, n, _ptr(Q), _ptr(dQ), _stream(stream)))
    return Q, dQ


def pxc_partition_function_noalloc(states: States, conds, stream=None):
    """Q[n_c], dQ[n_c, 2] and the device status word, with no workspace and no allocation in the library
    (the output tensors are the caller's).  At most 64 conditions; calls must not overlap on the GPU."""
    arr, n = _conds(conds)
    Q = torch.empty(n, dtype=torch.float64, device="cuda")
    dQ = torch.empty(n, 2, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = states.c()
    _check(load().pxc_partition_function_noalloc(ctypes.byref(st), arr, n, _ptr(Q), _ptr(dQ), _ptr(status),
                                                 _stream(stream)))
    return Q, dQ, status


def pxc_line_intensities(ws: Workspace, states: States, trans: Transitions, cond, grid=None, cutoff: float = 0.0,
                         threshold: float = 0.0, stream=None):
    """(nu[f64], I_scaled[f32], k[i32 scalar], n_kept[i64 scalar]) on the device."""
    n = trans.upper.numel()
    nu = torch.empty(n, dtype=torch.float64, device="cuda")
    Is = torch.empty(n, dtype=torch.float32, device="cuda")
    k = torch.empty(1, dtype=torch.int32, device="cuda")
    nk = torch.empty(1, dtype=torch.int64, device="cuda")
    arr, _ = _conds(cond)
    g = pxc_grid(*grid) if grid is not None else None
    st, tr = states.c(), trans.c()
    _check(load().pxc_line_intensities(ws.h, ctypes.byref(st), ctypes.byref(tr), arr,
                                       ctypes.byref(g) if g is not None else None, cutoff, threshold,
                                       _ptr(nu), _ptr(Is), _ptr(k), _ptr(nk), _stream(stream)))
    return nu, Is, k, nk


def pxc_cross_section(ws: Workspace, states: States, trans: Transitions, conds, grid, profile: Profile,
                      threshold: float = 0.0, sigma=None, sigma_exp=None, stream=None):
    """(sigma[n_c, n_grid] f32, exp[n_c] i32): sigma_phys = sigma * 2**exp."""
    arr, n_c = _conds(conds)
    ng = int(grid[2])
    if sigma is None:
        sigma = torch.empty(n_c, ng, dtype=torch.float32, device="cuda")
    if sigma_exp is None:
        sigma_exp = torch.empty(n_c, dtype=torch.int32, device="cuda")
    g = pxc_grid(*grid)
    st, tr, pa = states.c(), trans.c(), profile.c()
    _check(load().pxc_cross_section(ws.h, ctypes.byref(st), ctypes.byref(tr), arr, n_c, ctypes.byref(g),
                                    ctypes.byref(pa), threshold, _ptr(sigma), _ptr(sigma_exp), _stream(stream)))
    return sigma, sigma_exp


def pxc_cooling_function(ws: Workspace, states: States, trans: Transitions, conds, stream=None):
    """(W[n_c], Q[n_c]) float64 on the device: cooling functions, Eq. (cf)."""
    arr, n_c = _conds(conds)
    W = torch.empty(n_c, dtype=torch.float64, device="cuda")
    Q = torch.empty(n_c, dtype=torch.float64, device="cuda")
    st, tr = states.c(), trans.c()
    _check(load().pxc_cooling_function(ws.h, ctypes.byref(st), ctypes.byref(tr), arr, n_c, _ptr(W), _ptr(Q),
                                       _stream(stream)))
    return W, Q


def pxc_autotune(ws: Workspace, states: States, trans: Transitions, conds, grid, profile: Profile,
                 threshold: float = 0.0, repeats: int = 3, sigma=None, sigma_exp=None, stream=None):
    """Times every tile configuration on these inputs and keeps the fastest in the workspace.
    Returns (tile, [ms per call for each tile], sigma, exp); sigma/exp hold the chosen tile's result."""
    arr, n_c = _conds(conds)
    ng = int(grid[2])
    if sigma is None:
        sigma = torch.empty(n_c, ng, dtype=torch.float32, device="cuda")
    if sigma_exp is None:
        sigma_exp = torch.empty(n_c, dtype=torch.int32, device="cuda")
    g = pxc_grid(*grid)
    st, tr, pa = states.c(), trans.c(), profile.c()
    tile = c_i32(-1)
    ms = (ctypes.c_double * NUM_TILES)()
    _check(load().pxc_autotune(ws.h, ctypes.byref(st), ctypes.byref(tr), arr, n_c, ctypes.byref(g),
                               ctypes.byref(pa), threshold, _ptr(sigma), _ptr(sigma_exp), int(repeats),
                               ctypes.byref(tile), ms, _stream(stream)))
    return int(tile.value), list(ms), sigma, sigma_exp


def pxc_cross_section_backward(ws: Workspace, states: States, trans: Transitions, cond, grid, profile: Profile,
                               dL_dsigma: torch.Tensor, threshold: float = 0.0, stream=None):
    """Gradients of L(sigma_s) given dL/dsigma_s: dict of device tensors."""
    arr, n_c = _conds(cond)
    n = trans.upper.numel()
    out = {"dT": torch.zeros(1, dtype=torch.float64, device="cuda"),
           "dTvib": torch.zeros(1, dtype=torch.float64, device="cuda"),
           "dP": torch.zeros(1, dtype=torch.float64, device="cuda"),
           "dgamma_ref": torch.zeros(n, dtype=torch.float32, device="cuda"),
           "dA": torch.zeros(n, dtype=torch.float32, device="cuda")}
    g = pxc_grid(*grid)
    w = _dev(dL_dsigma.contiguous(), torch.float32, "dL_dsigma")
    st, tr, pa = states.c(), trans.c(), profile.c()
    _check(load().pxc_cross_section_backward(ws.h, ctypes.byref(st), ctypes.byref(tr), arr, n_c, ctypes.byref(g),
                                             ctypes.byref(pa), threshold, _ptr(w), _ptr(out["dT"]),
                                             _ptr(out["dTvib"]), _ptr(out["dP"]), _ptr(out["dgamma_ref"]),
                                             _ptr(out["dA"]), _stream(stream)))
    return out


def pxc_cross_section_streamed(ws: Workspace, states: States, upper, lower, A, gamma_ref, n_T, cond, grid,
                               profile: Profile, threshold: float = 0.0, bufs=None, sigma=None, sigma_exp=None,
                               stream=None):
    """Host-resident (preferably pinned) transition arrays streamed in chunks of the workspace's max_lines."""
    arr, _ = _conds(cond)
    L = load()
    broad = profile.kind in BROADENED
    a32 = int(A.dtype == torch.float32)
    nb = L.pxc_stream_buffer_bytes(ws.cap.max_lines, a32, int(broad))
    if bufs is None:
        bufs = (torch.empty(nb, dtype=torch.uint8, device="cuda"), torch.empty(nb, dtype=torch.uint8, device="cuda"))
    ng = int(grid[2])
    if sigma is None:
        sigma = torch.empty(ng, dtype=torch.float32, device="cuda")
    if sigma_exp is None:
        sigma_exp = torch.empty(1, dtype=torch.int32, device="cuda")
    g = pxc_grid(*grid)
    st, pa = states.c(), profile.c()
    for t in (upper, lower, A):
        if t.is_cuda:
            raise TypeError("streamed: transition arrays must be host tensors")
    _check(L.pxc_cross_section_streamed(ws.h, ctypes.byref(st), _ptr(upper), _ptr(lower), _ptr(A), a32,
                                        _ptr(gamma_ref) if broad else None, _ptr(n_T) if broad else None,
                                        upper.numel(), arr, ctypes.byref(g), ctypes.byref(pa), threshold,
                                        _ptr(bufs[0]), _ptr(bufs[1]), nb, _ptr(sigma), _ptr(sigma_exp),
                                        _stream(stream)))
    return sigma, sigma_exp, bufs


class CrossSection(torch.autograd.Function):
    """sigma_s(T, T_vib, P, gamma_ref, A) with the hand-written adjoint.

    forward(ws, states, upper, lower, grid, profile, threshold, T, T_vib, P, gamma_ref, A) -> (sigma_s, exp).
    T, T_vib, P are 0-d float64 tensors; gamma_ref, A per-line device tensors.  The exponent is held
    constant in the backward pass (sigma = sigma_s * 2**exp)."""

    @staticmethod
    def forward(ctx, ws, states, upper, lower, grid, profile, threshold, T, T_vib, P, gamma_ref, A):
        cond = (float(T), float(T_vib), float(P))
        prof = Profile(profile.kind, profile.cutoff, profile.mass_da, profile.hwhm, gamma_ref.detach(),
                       profile.n_T, profile.T_ref)
        tr = Transitions(upper, lower, A.detach())
        # the backward pass reads back this call's kept, sorted line list (same arrays by construction)
        ws.set_reuse_forward(True)
        sig, e = pxc_cross_section(ws, states, tr, cond, grid, prof, threshold)
        ctx.save_for_backward(T, T_vib, P, gamma_ref, A)
        ctx.ws, ctx.states, ctx.upper, ctx.lower, ctx.grid, ctx.profile, ctx.threshold = \
            ws, states, upper, lower, grid, profile, threshold
        ctx.mark_non_differentiable(e)
        return sig[0], e

    @staticmethod
    def backward(ctx, g_sigma, g_exp):
        T, T_vib, P, gamma_ref, A = ctx.saved_tensors
        prof = Profile(ctx.profile.kind, ctx.profile.cutoff, ctx.profile.mass_da, ctx.profile.hwhm,
                       gamma_ref.detach(), ctx.profile.n_T, ctx.profile.T_ref)
        tr = Transitions(ctx.upper, ctx.lower, A.detach())
        out = pxc_cross_section_backward(ctx.ws, ctx.states, tr, (float(T), float(T_vib), float(P)), ctx.grid,
                                         prof, g_sigma.float(), ctx.threshold)
        return (None, None, None, None, None, None, None,
                out["dT"][0].to(T.dtype), out["dTvib"][0].to(T_vib.dtype), out["dP"][0].to(P.dtype),
                out["dgamma_ref"].to(gamma_ref.dtype), out["dA"].to(A.dtype))
