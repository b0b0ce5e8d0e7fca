"""GPU parity of every profile-kernel tile configuration, and the autotuner.

Each tile (segment width 128 .. 2048 points) must give the oracle's sigma within
the same tolerances as the default, and the segment binning it reports must be
the oracle's binning for that width, bit for bit.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu

KINDS = {"gauss_doppler": 0, "gauss_hwhm": 1, "lorentz": 2, "voigt": 3}  # the binding's PROFILES


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def poly():
    return H.case("voigt_1e9", n_states=300_000, n_trans=40_000, hwhm=0.03, threshold=0.0)


@pytest.fixture(scope="module")
def poly_ref(poly):
    return {k: H.oracle_run(poly, kind=k, threshold=0.0)["sigma"] for k in KINDS}


def _ws(pxc, c, n_c=1, n_temps=0):
    w = c["w"]
    return pxc.Workspace(max_states=len(c["E"]), max_lines=max(len(c["up"]), 1), max_grid=w.n_grid,
                         max_conditions=n_c, max_temperatures=n_temps)


@pytest.mark.parametrize("kind", list(KINDS))
def test_every_tile_matches_oracle(pxc, poly, poly_ref, kind):
    w = poly["w"]
    ws = _ws(pxc, poly)
    st, tr, prof, grid = H.device(poly, kind)
    for tile in range(pxc.NUM_TILES):
        ws.set_tile(KINDS[kind], False, tile)
        assert ws.get_tile(KINDS[kind], False) == tile
        sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
        s = ws.stats()
        assert s["tile"] == tile and s["segment_points"] == pxc.TILE_SEGMENT_POINTS[tile]
        H.check_sigma(H.sigma_phys(sig[0], e[0].item()), poly_ref[kind], f"{kind} tile {tile}")


def test_every_tile_binning_bit_exact(pxc):
    c = H.case("doppler_1e5")
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c)
    r = H.oracle_run(c, with_sigma=False)
    ilo, ihi = r["ilo"][r["perm"]], r["ihi"][r["perm"]]
    for tile in range(pxc.NUM_TILES):
        ws.set_tile(0, False, tile)
        pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
        s = ws.stats()
        seg = pxc.TILE_SEGMENT_POINTS[tile]
        assert s["segment_points"] == seg and s["n_segments"] == -(-w.n_grid // seg)
        perm, first, last = ws.binning(s["n_kept"], s["n_segments"])
        assert np.array_equal(perm.cpu().numpy(), r["perm"])
        f_ref, l_ref = oracle.segment_ranges(ilo, ihi, w.n_grid, seg)
        assert np.array_equal(first.cpu().numpy(), f_ref), tile
        assert np.array_equal(last.cpu().numpy(), l_ref), tile


@pytest.mark.parametrize("tile", [0, 2])
def test_batched_table_on_narrow_tiles(pxc, poly, tile):
    w = poly["w"]
    conds = [(T, 0.0, P) for T in (300.0, 3000.0) for P in (1e-3, 1.0)]
    ws = _ws(pxc, poly, n_c=len(conds), n_temps=2)
    ws.set_tile(3, True, tile)
    st, tr, prof, grid = H.device(poly)
    sig, e = pxc.pxc_cross_section(ws, st, tr, conds, grid, prof)
    assert ws.stats()["tile"] == tile
    for i, (T, _, P) in enumerate(conds):
        r = H.oracle_run(poly, T=T, P=P, threshold=0.0)
        H.check_sigma(H.sigma_phys(sig[i], e[i].item()), r["sigma"], f"batched tile {tile} T={T} P={P}")


def test_autotune_picks_a_tile_and_keeps_result(pxc, poly, poly_ref):
    w = poly["w"]
    ws = _ws(pxc, poly)
    st, tr, prof, grid = H.device(poly)
    tile, ms, sig, e = pxc.pxc_autotune(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0, repeats=2)
    assert 0 <= tile < pxc.NUM_TILES
    assert all(m > 0 for m in ms) and ms[tile] == min(ms)
    assert ws.get_tile(3, False) == tile
    assert ws.get_tile(3, True) == pxc.BATCHED_DEFAULT_TILE  # the batched choice is untouched
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), poly_ref["voigt"], "autotuned")
    # the next plain call uses the chosen tile
    pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
    assert ws.stats()["tile"] == tile


def test_tile_arguments_checked(pxc, poly):
    ws = _ws(pxc, poly)
    for args in [(11, False, 0), (-1, False, 0), (0, False, pxc.NUM_TILES), (0, False, -1)]:
        with pytest.raises(pxc.PxcError) as ei:
            ws.set_tile(*args)
        assert ei.value.code == 1
    ws.set_accumulate(True)
    w = poly["w"]
    st, tr, prof, grid = H.device(poly)
    with pytest.raises(pxc.PxcError):
        pxc.pxc_autotune(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
    ws.set_accumulate(False)
