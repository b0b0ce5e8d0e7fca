"""GPU parity for the pseudo-Voigt profiles and for wavelength grids (Table profile; Sec. 2.4.3).

Pseudo-Voigt kinds (Thompson, Olivero, Liu-Lin) on the polyatomic list against the oracle, on
every tile configuration for one of them.  Wavelength grids (nm and um) with the sampled kinds:
the kept set, the line order (descending nu, ties by index) and the segment binning bit-exact,
sigma within the usual tolerances, single and batched calls; the kinds and calls that do not
take a wavelength grid are refused on the host.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu
PV = ["pv_thompson", "pv_olivero", "pv_liulin"]


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def poly():
    return H.case("voigt_1e9", n_states=300_000, n_trans=40_000, threshold=0.0)


def _ws(pxc, c, n_c=1, n_grid=None):
    return pxc.Workspace(max_states=len(c["E"]), max_lines=len(c["up"]), max_grid=n_grid or c["w"].n_grid,
                         max_conditions=n_c)


@pytest.mark.parametrize("kind", PV)
def test_pseudo_voigt_against_oracle(pxc, poly, kind):
    c = poly
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, kind)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    ws.sync()
    r = H.oracle_run(c, kind=kind, threshold=0.0)
    assert int(e[0].item()) == r["k"]
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], kind)


def test_pseudo_voigt_every_tile(pxc, poly):
    c = poly
    w = c["w"]
    st, tr, prof, grid = H.device(c, "pv_olivero")
    r = H.oracle_run(c, kind="pv_olivero", threshold=0.0)
    for tile in range(pxc.NUM_TILES):
        ws = _ws(pxc, c)
        ws.set_tile(pxc.PROFILES["pv_olivero"], False, tile)
        sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
        ws.sync()
        H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], f"pv_olivero tile {tile}")


def _wl_case(unit, n_trans=30_000):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=n_trans, threshold=0.0)
    if unit == 1e7:
        lam0, dlam, n = 500.0, 0.01, 450_001       # 500 .. 5000 nm: 20000 .. 2000 cm^-1
    else:
        lam0, dlam, n = 0.5, 1e-5, 450_001          # the same points in um
    return c, (lam0, dlam, n, unit)


@pytest.mark.parametrize("kind", ["voigt", "gauss_doppler", "lorentz", "pv_liulin"])
def test_wavelength_grid_nm(pxc, kind):
    c, grid = _wl_case(1e7)
    w = c["w"]
    st, tr, prof, _ = H.device(c, kind)
    ws = _ws(pxc, c, n_grid=grid[2])
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    s = ws.stats()
    r = oracle.run(c["E"], c["g"], None, c["up"], c["lo"], c["A"], c["gr"], c["ne"], kind=kind, T=w.T, P=w.P,
                   mass_da=w.mass_da, nu_min=grid[0], dnu=grid[1], n_grid=grid[2], cut=w.cutoff, wl_unit=grid[3])
    assert s["n_kept"] == int(r["keep"].sum())
    assert int(e[0].item()) == r["k"]
    perm, first, last = ws.binning(s["n_kept"], s["n_segments"])
    assert np.array_equal(perm.cpu().numpy(), r["perm"]), "descending nu, ties by index"
    f_ref, l_ref = oracle.segment_ranges(r["ilo"][r["perm"]], r["ihi"][r["perm"]], grid[2], s["segment_points"])
    assert np.array_equal(first.cpu().numpy(), f_ref) and np.array_equal(last.cpu().numpy(), l_ref)
    assert s["evals_window"] == r["evals"]
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], f"{kind} on a nm grid")


def test_wavelength_grid_um_batched_and_stick(pxc):
    import torch
    c, grid = _wl_case(1e4, n_trans=20_000)
    w = c["w"]
    st, tr, prof, _ = H.device(c, "voigt")
    conds = [(w.T, 0.0, w.P), (700.0, 0.0, 3.0)]
    ws = _ws(pxc, c, n_c=2, n_grid=grid[2])
    sig, e = pxc.pxc_cross_section(ws, st, tr, conds, grid, prof)
    ws.sync()
    for j, (T, _, P) in enumerate(conds):
        r = oracle.run(c["E"], c["g"], None, c["up"], c["lo"], c["A"], c["gr"], c["ne"], kind="voigt", T=T, P=P,
                       mass_da=w.mass_da, nu_min=grid[0], dnu=grid[1], n_grid=grid[2], cut=w.cutoff,
                       wl_unit=grid[3])
        H.check_sigma(H.sigma_phys(sig[j], e[j].item()), r["sigma"], f"um grid, T={T}")
    # stick spectrum on the wavelength grid: the kept set follows the wavelength windows
    nu, Is, k, nk = pxc.pxc_line_intensities(ws, st, tr, conds[0], grid, w.cutoff, 0.0)
    ws.sync()
    r = oracle.run(c["E"], c["g"], None, c["up"], c["lo"], c["A"], c["gr"], c["ne"], kind="voigt", T=w.T, P=w.P,
                   mass_da=w.mass_da, nu_min=grid[0], dnu=grid[1], n_grid=grid[2], cut=w.cutoff, wl_unit=grid[3],
                   with_sigma=False)
    assert int(nk.item()) == int(r["keep"].sum()) and int(k.item()) == r["k"]
    assert np.array_equal(Is.cpu().numpy() != 0, r["I_s"] != 0)
    del torch


def test_refused_combinations(pxc, poly):
    c = poly
    w = c["w"]
    st, tr, prof, grid = H.device(c, "binned_voigt")
    ws = _ws(pxc, c, n_grid=1000)
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), (1000.0, 0.01, 1000, 1e7), prof)
    assert ei.value.code == 1
    st, tr, prof, grid = H.device(c, "voigt")
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), (1000.0, 0.01, 1000, -1.0), prof)
    assert ei.value.code == 1
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), (0.0, 0.01, 1000, 1e7), prof)  # lambda_min = 0
    assert ei.value.code == 1
    import torch
    wgt = torch.ones(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section_backward(ws, st, tr, (w.T, 0.0, w.P), (1000.0, 0.01, 1000, 1e7), prof, wgt)
    assert ei.value.code == 1
    st, tr, prof, _ = H.device(c, "pv_olivero")
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section_backward(ws, st, tr, (w.T, 0.0, w.P), (1000.0, 0.01, 1000), prof, wgt)
    assert ei.value.code == 1
