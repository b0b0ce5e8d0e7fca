"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bit-exact: nu, the kept-line set, the list exponent, the sorted line order and
the segment binning.  Floating point: FP32 scaled intensities within 1 ulp of
the oracle's rounding of ldexp(I, -k); sigma within 1e-4 of its peak and 1e-3
per bin wherever sigma > 1e-6 of the peak (tests/helpers.py).
"""
import math

import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


def _ws(pxc, c, n_c=1, n_temps=0):
    w = c["w"]
    return pxc.Workspace(max_states=len(c["E"]), max_lines=max(len(c["up"]), 1), max_grid=w.n_grid,
                         max_conditions=n_c, max_temperatures=n_temps)


# ------------------------------------------------------------------ partition functions

def test_partition_function_lte_and_two_temperature(pxc):
    import torch
    c = H.case("doppler_1e5")
    ws = _ws(pxc, c, n_c=4)
    st, _, _, _ = H.device(c)
    conds = [(296.0, 0.0, 1.0), (1000.0, 0.0, 1.0), (3000.0, 0.0, 1.0), (1200.0, 2500.0, 1.0)]
    Q, dQ = pxc.pxc_partition_function(ws, st, conds)
    ws.sync()
    for i, (T, Tv, _) in enumerate(conds):
        ref = oracle.partition(c["E"], c["g"], c["Ev"] if Tv > 0 else None, T, Tv)
        assert Q[i].item() == pytest.approx(ref[0], rel=1e-12)
        assert dQ[i, 0].item() == pytest.approx(ref[1], rel=1e-10)
        if Tv > 0:
            assert dQ[i, 1].item() == pytest.approx(ref[2], rel=1e-10)
    del torch


# ------------------------------------------------------------------ intensities

@pytest.mark.parametrize("name,kw", [("doppler_1e5", {}),
                                     ("nlte_1e7", dict(n_trans=200_000)),
                                     ("voigt_1e9", dict(n_states=400_000, n_trans=300_000))])
def test_line_intensities_bit_exact_nu_and_kept_set(pxc, name, kw):
    c = H.case(name, **kw)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, _, grid = H.device(c)
    nu, Is, k, nk = pxc.pxc_line_intensities(ws, st, tr, (w.T, w.T_vib, w.P), grid, w.cutoff, w.threshold)
    ws.sync()
    r = H.oracle_run(c, with_sigma=False)
    nu_g = nu.cpu().numpy()
    assert np.array_equal(nu_g.view(np.uint64), r["nu"].view(np.uint64)), "nu must be bit-exact"
    keep = r["keep"].astype(bool)
    if w.threshold > 0:
        band = keep & (np.abs(r["I"] / w.threshold - 1.0) < 1e-9)
        assert not band.any(), "fixture has lines within the threshold rounding band"
    assert int(nk.item()) == int(keep.sum())
    assert int(k.item()) == r["k"]
    Ig = Is.cpu().numpy()
    Io = r["I_s"]
    ulp = np.spacing(np.abs(Io).astype(np.float32)).astype(np.float64)
    d = np.abs(Ig.astype(np.float64) - Io.astype(np.float64))
    assert np.all(d <= ulp), f"I_s off by more than 1 ulp on {(d > ulp).sum()} lines"


# ------------------------------------------------------------------ sorting and binning

def test_sorted_order_and_segment_binning_bit_exact(pxc):
    c = H.case("doppler_1e5")
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    s = ws.stats()
    r = H.oracle_run(c, with_sigma=False)
    perm, first, last = ws.binning(s["n_kept"], s["n_segments"])
    assert np.array_equal(perm.cpu().numpy(), r["perm"])
    f_ref, l_ref = oracle.segment_ranges(r["ilo"][r["perm"]], r["ihi"][r["perm"]], w.n_grid, s["segment_points"])
    assert np.array_equal(first.cpu().numpy(), f_ref) and np.array_equal(last.cpu().numpy(), l_ref)
    assert s["evals_window"] == r["evals"]


def test_duplicate_nu_ties_broken_by_index(pxc):
    import torch
    # many transitions with identical nu (the same pair repeated) and a few distinct ones
    E = np.array([0.0, 100.0, 250.0, 100.0], np.float64)
    g = np.array([1, 3, 5, 3], np.int32)
    up = np.array([1, 2, 3, 1, 2, 3, 1, 3, 2, 1] * 50, np.int32)
    lo = np.zeros(up.size, np.int32)
    A = np.linspace(1.0, 2.0, up.size)
    c = {"w": H.synth.workload("doppler_1e5").scaled(n_trans=up.size, n_states=4, nu_min=0.0, dnu=0.5,
                                                      n_grid=1000, T=500.0),
         "E": E, "g": g, "Ev": np.zeros(4), "up": up, "lo": lo, "A": A,
         "gr": np.full(up.size, 0.05, np.float32), "ne": np.full(up.size, 0.5, np.float32)}
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (500.0, 0.0, 1.0), grid, prof)
    s = ws.stats()
    perm, _, _ = ws.binning(s["n_kept"], s["n_segments"])
    r = H.oracle_run(c)
    assert np.array_equal(perm.cpu().numpy(), r["perm"])
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "ties")
    del torch


# ------------------------------------------------------------------ cross sections

def test_cross_section_doppler_full_size(pxc):
    c = H.case("doppler_1e5")
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    assert int(e[0].item()) == r["k"]
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "doppler_1e5")


@pytest.mark.parametrize("kind", ["voigt", "lorentz", "gauss_hwhm", "gauss_doppler"])
def test_cross_section_profiles_polyatomic(pxc, kind):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=40_000, hwhm=0.03, threshold=0.0)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, kind)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
    ws.sync()
    r = H.oracle_run(c, kind=kind, threshold=0.0)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], kind)


def test_cross_section_voigt_threshold(pxc):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=60_000)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    s = ws.stats()
    r = H.oracle_run(c)
    assert s["n_kept"] == int(r["keep"].sum())
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "voigt threshold")


def test_cross_section_voigt_diatomic_subset(pxc):
    c = H.case("voigt_1e7", n_trans=150_000)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "voigt_1e7 subset")


def test_cross_section_two_temperature(pxc):
    c = H.case("nlte_1e7", n_trans=150_000)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, w.T_vib, w.P), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "nlte")


def test_batched_table_matches_oracle_and_plain(pxc):
    c = H.case("voigt_1e9", n_states=200_000, n_trans=20_000, threshold=0.0)
    w = c["w"]
    conds = [(T, 0.0, P) for T in (300.0, 1200.0, 3000.0) for P in (1e-3, 1.0)]
    ws = _ws(pxc, c, n_c=len(conds), n_temps=3)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, conds, grid, prof)
    ws.sync()
    ws1 = _ws(pxc, c)
    for i, (T, _, P) in enumerate(conds):
        r = H.oracle_run(c, T=T, P=P, threshold=0.0)
        got = H.sigma_phys(sig[i], e[i].item())
        H.check_sigma(got, r["sigma"], f"batched T={T} P={P}")
        s1, e1 = pxc.pxc_cross_section(ws1, st, tr, (T, 0.0, P), grid, prof)
        plain = H.sigma_phys(s1[0], e1[0].item())
        assert np.max(np.abs(plain - got)) <= 1e-5 * plain.max()


def test_batched_table_with_split_segments_matches_plain(pxc):
    # enough lines that single-condition calls split dense segments into several items;
    # the batched call must cover every line of every segment all the same
    c = H.case("table_1e8", n_trans=3_000_000)
    conds = [(200.0, 0.0, 1e-5), (1000.0, 0.0, 1.0), (3000.0, 0.0, 100.0)]
    ws = _ws(pxc, c, n_c=len(conds), n_temps=3)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, conds, grid, prof)
    ws1 = _ws(pxc, c)
    for i, cond in enumerate(conds):
        s1, e1 = pxc.pxc_cross_section(ws1, st, tr, cond, grid, prof)
        plain = H.sigma_phys(s1[0], e1[0].item())
        got = H.sigma_phys(sig[i], e[i].item())
        assert np.max(np.abs(plain - got)) <= 1e-5 * np.abs(plain).max(), cond
    ws.sync()


def test_streamed_chunks_match_single_call(pxc):
    import torch
    c = H.case("voigt_1e9", n_states=200_000, n_trans=30_000)
    w = c["w"]
    st, tr, prof, grid = H.device(c)
    ws1 = _ws(pxc, c)
    s1, e1 = pxc.pxc_cross_section(ws1, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    one = H.sigma_phys(s1[0], e1[0].item())
    wsc = pxc.Workspace(max_states=len(c["E"]), max_lines=7_000, max_grid=w.n_grid)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    sig, e, _ = pxc.pxc_cross_section_streamed(wsc, st, pin(c["up"]), pin(c["lo"]), pin(c["A"]), pin(c["gr"]),
                                               pin(c["ne"]), (w.T, 0.0, w.P), grid, prof, w.threshold)
    wsc.sync()
    got = H.sigma_phys(sig, e.item())
    assert np.max(np.abs(got - one)) <= 1e-5 * one.max()
    r = H.oracle_run(c)
    H.check_sigma(got, r["sigma"], "streamed")


def test_deterministic_replay(pxc):
    c = H.case("voigt_1e9", n_states=200_000, n_trans=30_000)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    a, ea = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    a = a.clone()
    b, eb = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    assert int(ea.item()) == int(eb.item())
    assert bool((a == b).all())


# ------------------------------------------------------------------ edge cases and errors

def test_edge_cases_empty_tiny_and_offgrid(pxc):
    import torch
    w = H.synth.workload("doppler_1e5").scaled(nu_min=100.0, dnu=0.5, n_grid=401, cutoff=5.0, T=800.0)
    # states so that nu covers: negative, zero, below the grid with wings inside, exactly nu_min - cut,
    # above the grid with wings inside, far off-grid
    E = np.array([0.0, 96.0, 95.0, 300.5, 304.0, 350.0, 50.0, 150.0, 150.0], np.float64)
    g = np.arange(1, 10, dtype=np.int32)
    up = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 7], np.int32)
    lo = np.array([1, 0, 0, 0, 0, 0, 0, 0, 0, 8], np.int32)
    A = np.full(up.size, 3.0)
    c = {"w": w.scaled(n_states=E.size, n_trans=up.size), "E": E, "g": g, "Ev": np.zeros(E.size), "up": up,
         "lo": lo, "A": A, "gr": np.full(up.size, 0.05, np.float32), "ne": np.full(up.size, 0.5, np.float32)}
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (800.0, 0.0, 1.0), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    s = ws.stats()
    assert s["n_kept"] == int(r["keep"].sum())
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "edge")
    # 1e-50-scale intensities: same sigma shape, exponent shifted, no underflow
    c2 = dict(c); c2["A"] = A * 1e-45
    st2, tr2, prof2, _ = H.device(c2)
    sig2, e2 = pxc.pxc_cross_section(ws, st2, tr2, (800.0, 0.0, 1.0), grid, prof2)
    ws.sync()
    r2 = H.oracle_run(c2)
    assert r2["I"].max() < 1e-50
    H.check_sigma(H.sigma_phys(sig2[0], e2[0].item()), r2["sigma"], "tiny intensities")
    # empty list
    c3 = dict(c); c3["up"] = up[:0]; c3["lo"] = lo[:0]; c3["A"] = A[:0]
    c3["gr"] = c["gr"][:0]; c3["ne"] = c["ne"][:0]
    st3, tr3, prof3, _ = H.device(c3)
    sig3, e3 = pxc.pxc_cross_section(ws, st3, tr3, (800.0, 0.0, 1.0), grid, prof3)
    ws.sync()
    assert float(sig3.abs().max()) == 0.0
    del torch


def test_error_statuses(pxc):
    import torch
    c = H.case("doppler_1e5", n_trans=5000)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    bad = pxc.Transitions(tr.upper.clone(), tr.lower, tr.A)
    bad.upper[17] = len(c["E"])  # out of range
    pxc.pxc_cross_section(ws, st, bad, (w.T, 0.0, w.P), grid, prof)
    with pytest.raises(pxc.PxcError) as ei:
        ws.sync()
    assert ei.value.code == 2
    nanA = pxc.Transitions(tr.upper, tr.lower, tr.A.clone())
    nanA.A[3] = float("inf")
    pxc.pxc_cross_section(ws, st, nanA, (w.T, 0.0, w.P), grid, prof)
    with pytest.raises(pxc.PxcError) as ei:
        ws.sync()
    assert ei.value.code == 3
    El, gl, _ = w.states(literal=True)
    stl = pxc.States(torch.from_numpy(El).cuda(), torch.from_numpy(gl).cuda(), None)
    pxc.pxc_cross_section(ws, stl, tr, (w.T, 0.0, w.P), grid, prof)
    with pytest.raises(pxc.PxcError) as ei:
        ws.sync()
    assert ei.value.code == 4
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(ws, st, tr, (-5.0, 0.0, w.P), grid, prof)
    assert ei.value.code == 1
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), (0.0, 0.0, 10), prof)
    assert ei.value.code == 1
    small = pxc.Workspace(max_states=len(c["E"]), max_lines=100, max_grid=w.n_grid)
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(small, st, tr, (w.T, 0.0, w.P), grid, prof)
    assert ei.value.code == 7
    # the workspace stays usable after errors
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "after errors")


# ------------------------------------------------------------------ full size, sampled

def test_full_size_chunk_sampled_windows(pxc):
    """One 1e8-line chunk of the 1e9-line Voigt workload (5e7 states), in the launch
    configuration the benchmark times, checked on sampled grid windows."""
    import torch
    w = H.synth.workload("voigt_1e9")
    E, g, Ev = w.states()
    up, lo, A = w.transitions(0, w.chunk)
    gr, ne = w.broadening(0, w.chunk)
    ws = pxc.Workspace(max_states=w.n_states, max_lines=w.chunk, max_grid=w.n_grid)
    st = pxc.States(torch.from_numpy(E).cuda(), torch.from_numpy(g).cuda(), None)
    tr = pxc.Transitions(torch.from_numpy(up).cuda(), torch.from_numpy(lo).cuda(), torch.from_numpy(A).cuda())
    prof = pxc.Profile("voigt", w.cutoff, w.mass_da, 0.0, torch.from_numpy(gr).cuda(), torch.from_numpy(ne).cuda())
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), (w.nu_min, w.dnu, w.n_grid), prof, w.threshold)
    s = ws.stats()
    got_all = H.sigma_phys(sig[0], e[0].item())
    Q = oracle.partition(E, g, None, w.T)
    nu, I, keep, ilo, ihi = oracle.line_intensities(E, g, None, up, lo, A, w.T, 0.0, Q[0], w.nu_min, w.dnu,
                                                    w.n_grid, w.cutoff, w.threshold)
    assert s["n_kept"] == int(keep.sum())
    assert int(e[0].item()) == oracle.list_exponent(I, keep)
    rng = np.random.default_rng(w.seed)
    starts = sorted(rng.integers(0, w.n_grid - 300, 6).tolist()) + [w.n_grid - 300]
    for i0 in starts:
        m = 300
        sel = keep.astype(bool) & (ihi >= i0) & (ilo <= i0 + m - 1)
        idx = np.nonzero(sel)[0]
        alpha, gamma = oracle.widths("voigt", nu[idx], gr[idx], ne[idx], w.T, w.P, w.mass_da)
        ref = oracle.cross_section_window("voigt", nu[idx], I[idx], alpha, gamma, keep[idx], ilo[idx], ihi[idx],
                                          w.nu_min, w.dnu, i0, m)
        got = got_all[i0:i0 + m]
        if ref.max() == 0:
            assert np.all(got == 0)
            continue
        d = np.abs(got - ref)
        peak = max(ref.max(), 1e-300)
        big = ref > 1e-6 * peak
        assert np.all(d[big] / ref[big] <= H.SIG_REL), f"window {i0}: {np.max(d[big] / ref[big])}"
    del torch


# ------------------------------------------------------------------ state-code prefilter edges

def _edge_case(rng_seed, threshold_quantile, E_offset):
    """States in pairs whose nu lands within +-0.05 cm^-1 of the kept window's ends (and spread
    over it), plus random pairs; threshold at a quantile of |I| so many lines sit near it."""
    rng = np.random.default_rng(rng_seed)
    n_pair = 6000
    w = H.synth.workload("doppler_1e5").scaled(n_states=2 * n_pair + 4000, n_trans=0, nu_min=1000.0, dnu=0.01,
                                                n_grid=100_001, T=900.0, cutoff=5.0, threshold=0.0)
    lo_edge, hi_edge = w.nu_min - w.cutoff, w.nu_min + (w.n_grid - 1) * w.dnu + w.cutoff
    targets = np.concatenate([lo_edge + rng.uniform(-0.05, 0.05, n_pair // 3),
                              hi_edge + rng.uniform(-0.05, 0.05, n_pair // 3),
                              rng.uniform(lo_edge - 50.0, hi_edge + 50.0, n_pair - 2 * (n_pair // 3))])
    El = rng.uniform(0.0, 40000.0, n_pair) + E_offset
    E = np.empty(w.n_states)
    E[0:2 * n_pair:2] = El
    E[1:2 * n_pair:2] = El + targets
    E[2 * n_pair:] = rng.uniform(0.0, 45000.0, w.n_states - 2 * n_pair) + E_offset
    g = rng.integers(1, 60, w.n_states).astype(np.int32)
    up = np.concatenate([np.arange(1, 2 * n_pair, 2), rng.integers(0, w.n_states, 30000)]).astype(np.int32)
    lo = np.concatenate([np.arange(0, 2 * n_pair, 2), rng.integers(0, w.n_states, 30000)]).astype(np.int32)
    A = 10.0 ** rng.uniform(-6, 2, up.size)
    c = {"w": w.scaled(n_trans=up.size), "E": E, "g": g, "Ev": np.zeros(w.n_states), "up": up, "lo": lo, "A": A,
         "gr": np.full(up.size, 0.05, np.float32), "ne": np.full(up.size, 0.5, np.float32)}
    if threshold_quantile is not None:
        r0 = H.oracle_run(c, threshold=0.0, with_sigma=False)
        Ik = np.sort(np.abs(r0["I"][r0["keep"].astype(bool)]))
        j = int(threshold_quantile * (Ik.size - 1))
        while Ik[j + 1] <= Ik[j] * (1 + 1e-6):  # no line within rounding of the threshold
            j += 1
        c["w"] = c["w"].scaled(threshold=float(np.sqrt(Ik[j] * Ik[j + 1])))
    return c


@pytest.mark.parametrize("seed,q,off", [(1, None, 0.0), (2, 0.5, 0.0), (3, 0.9, -75.0), (4, 0.2, 1234.5)])
def test_prefilter_keeps_exact_set_at_window_and_threshold_edges(pxc, seed, q, off):
    c = _edge_case(seed, q, off)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    s = ws.stats()
    r = H.oracle_run(c)
    keep = r["keep"].astype(bool)
    assert s["n_kept"] == int(keep.sum())
    perm, _, _ = ws.binning(s["n_kept"], s["n_segments"])
    assert np.array_equal(perm.cpu().numpy(), r["perm"])
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], f"prefilter edges {seed}")


def test_lines_near_zero_wavenumber(pxc):
    """Lines with nu from 5e-4 to 30 cm^-1 on a grid starting at 0: the Doppler width is at its
    floor and one grid step spans up to ~1e5 Doppler widths, so every profile path meets |x| up to
    ~1e8 (and |x| + y < 15 near the centre at low pressure).  sigma stays finite and matches."""
    E = np.array([0.0, 0.0005, 0.0013, 0.02, 0.2, 3.0, 30.0])
    g = np.array([1, 3, 5, 3, 5, 7, 9], np.int32)
    up = np.arange(1, E.size, dtype=np.int32)
    lo = np.zeros(up.size, np.int32)
    A = np.full(up.size, 1e-3)
    w = H.synth.workload("voigt_1e9").scaled(n_states=E.size, n_trans=up.size, nu_min=0.0, dnu=0.01, n_grid=100_001,
                                              T=2000.0, threshold=0.0)
    c = {"w": w, "E": E, "g": g, "Ev": np.zeros(E.size), "up": up, "lo": lo, "A": A,
         "gr": np.full(up.size, 0.05, np.float32), "ne": np.full(up.size, 0.5, np.float32)}
    st, tr, _, grid = H.device(c)
    for kind in ("voigt", "lorentz", "gauss_doppler"):
        _, _, prof, _ = H.device(c, kind)
        for P in (1e-5, 1e-2, 1.0):
            for tile in range(pxc.NUM_TILES):
                ws = _ws(pxc, c)
                ws.set_tile(pxc.PROFILES[kind], False, tile)
                sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, P), grid, prof)
                ws.sync()
                got = H.sigma_phys(sig[0], e[0].item())
                assert np.isfinite(got).all(), (kind, P, tile)
                r = H.oracle_run(c, kind=kind, P=P, threshold=0.0)
                H.check_sigma(got, r["sigma"], f"{kind} P={P} tile {tile}")
