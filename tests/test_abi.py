"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/pxc.h declares, and its host-only argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pxc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pxc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_17273_b300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_library_exports_every_declared_function(lib):
    L, path = lib
    names = _declared()
    assert "pxc_cross_section" in names and "pxc_partition_function" in names
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pxc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        getattr(L, n)


def test_binding_names_match_header():
    import paper_2609_17273_b300 as pxc
    assert sorted(pxc.ABI_FUNCTIONS) == _declared()


def test_host_side_argument_checks_without_gpu(lib):
    import paper_2609_17273_b300 as pxc
    L = pxc.load()
    cap = pxc.pxc_capacity(1000, 1000, 5000, 1, 0)
    nb = ctypes.c_size_t()
    assert L.pxc_workspace_query(ctypes.byref(cap), ctypes.byref(nb)) == 0
    assert nb.value > 1000 * 50
    bad = pxc.pxc_capacity(-1, 1000, 5000, 1, 0)
    assert L.pxc_workspace_query(ctypes.byref(bad), ctypes.byref(nb)) == 1
    assert b"bad capacity" in L.pxc_last_error()
    h = ctypes.c_void_p()
    # null scratch buffer is rejected before any CUDA call
    assert L.pxc_workspace_create(ctypes.byref(cap), None, nb.value, ctypes.byref(h)) == 1
    # misaligned buffer
    assert L.pxc_workspace_create(ctypes.byref(cap), ctypes.c_void_p(0x1001), nb.value, ctypes.byref(h)) == 1
    assert L.pxc_stream_buffer_bytes(1000, 1, 1) >= 1000 * 20


def test_workspace_grows_linearly_with_lines(lib):
    import paper_2609_17273_b300 as pxc
    L = pxc.load()
    sizes = []
    for n in (10**6, 2 * 10**6):
        cap = pxc.pxc_capacity(10**5, n, 10**6, 1, 0)
        nb = ctypes.c_size_t()
        assert L.pxc_workspace_query(ctypes.byref(cap), ctypes.byref(nb)) == 0
        sizes.append(nb.value)
    per_line = (sizes[1] - sizes[0]) / 1e6
    assert 60 < per_line < 200, per_line


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2609_17273_b300 as pxc
    saved = pxc._lib
    pxc._lib = None
    try:
        with pytest.raises(ImportError):
            pxc.load(str(tmp_path / "missing.so"))
    finally:
        pxc._lib = saved


def test_null_workspace_and_bad_arguments_are_rejected_on_the_host(lib):
    # every entry point checks its arguments before touching the device
    import paper_2609_17273_b300 as pxc
    L = pxc.load()
    assert L.pxc_set_tile(None, 3, 0, 0) == 1
    assert L.pxc_get_tile(None, 3, 0, None) == 1
    assert L.pxc_set_emission(None, 1) == 1
    assert L.pxc_set_wait_limit(None, 10) == 1
    assert L.pxc_set_accumulate(None, 1) == 1
    assert L.pxc_cooling_function(None, None, None, None, 1, None, None, None) == 1
    assert L.pxc_cross_section(None, None, None, None, 1, None, None, 0.0, None, None, None) == 1
    assert L.pxc_partition_function_noalloc(None, None, 1, None, None, None, None) == 1
    cond = (pxc.pxc_condition * 65)()
    st = pxc.pxc_states(ctypes.c_void_p(16), ctypes.c_void_p(16), None, 10, None)
    for i in range(65):
        cond[i] = pxc.pxc_condition(300.0, 0.0, 1.0)
    # more conditions than the fixed scratch holds: a capacity error, still on the host
    assert L.pxc_partition_function_noalloc(ctypes.byref(st), cond, 65, ctypes.c_void_p(16), None, None,
                                            None) == 7
    assert b"64" in L.pxc_last_error()


def test_noalloc_rejects_what_the_workspace_entry_point_rejects(lib):
    # the allocation-free partition function runs the same host-side checks as
    # pxc_partition_function, before any CUDA call
    import paper_2609_17273_b300 as pxc
    L = pxc.load()
    st = pxc.pxc_states(ctypes.c_void_p(16), ctypes.c_void_p(16), None, 10, None)
    Q = ctypes.c_void_p(16)
    for T, Tv in [(float("inf"), 0.0), (float("nan"), 0.0), (0.0, 0.0), (-300.0, 0.0), (300.0, float("nan")),
                  (300.0, float("inf")), (300.0, 2500.0)]:   # the last needs E_vib
        cond = pxc.pxc_condition(T, Tv, 1.0)
        assert L.pxc_partition_function_noalloc(ctypes.byref(st), ctypes.byref(cond), 1, Q, None, None, None) == 1, \
            (T, Tv)
    # vibronic densities need E_vib and exclude T_vib
    dens = pxc.pxc_states(ctypes.c_void_p(16), ctypes.c_void_p(16), None, 10, ctypes.c_void_p(16))
    cond = pxc.pxc_condition(300.0, 0.0, 1.0)
    assert L.pxc_partition_function_noalloc(ctypes.byref(dens), ctypes.byref(cond), 1, Q, None, None, None) == 1
    # more states than the 32-bit state ids can address
    big = pxc.pxc_states(ctypes.c_void_p(16), ctypes.c_void_p(16), None, 2 ** 31, None)
    assert L.pxc_partition_function_noalloc(ctypes.byref(big), ctypes.byref(cond), 1, Q, None, None, None) == 1
    assert b"2^31" in L.pxc_last_error()
    neg = pxc.pxc_states(ctypes.c_void_p(16), ctypes.c_void_p(16), None, -1, None)
    assert L.pxc_partition_function_noalloc(ctypes.byref(neg), ctypes.byref(cond), 1, Q, None, None, None) == 1
