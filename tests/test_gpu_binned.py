"""GPU parity of the binned profiles (bin averages over the grid bins, Table profile) against
the FP64 oracle, with the same sigma tolerances as the sampled profiles, and the property that
makes them worth having: on a grid too coarse to sample the Doppler cores, sum(sigma) dnu still
equals the sum of the kept intensities."""
import numpy as np
import pytest

from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


def _ws(pxc, c):
    w = c["w"]
    return pxc.Workspace(max_states=len(c["E"]), max_lines=max(len(c["up"]), 1), max_grid=w.n_grid)


@pytest.mark.parametrize("kind", ["binned_gauss_doppler", "binned_gauss_hwhm", "binned_lorentz", "binned_voigt"])
def test_binned_polyatomic_fine_grid(pxc, kind):
    n = 1000 if kind == "binned_voigt" else 40_000
    c = H.case("voigt_1e9", n_states=300_000, n_trans=n, hwhm=0.03, threshold=0.0)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, kind)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
    r = H.oracle_run(c, kind=kind, threshold=0.0)
    assert int(e[0].item()) == r["k"]
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], kind)


@pytest.mark.parametrize("kind", ["binned_gauss_doppler", "binned_voigt", "binned_lorentz"])
def test_binned_coarse_grid_narrow_lines(pxc, kind):
    # doppler_1e5: 0.1 cm^-1 bins, Doppler HWHM ~1e-3..2e-2 cm^-1 (undersampled when sampled)
    n = 5000 if kind == "binned_voigt" else None
    c = H.case("doppler_1e5", n_trans=n) if n else H.case("doppler_1e5")
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, kind)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    r = H.oracle_run(c, kind=kind)
    got = H.sigma_phys(sig[0], e[0].item())
    H.check_sigma(got, r["sigma"], kind)
    if kind == "binned_gauss_doppler":
        # lines whose +-25 cm^-1 window lies inside the grid keep all their intensity
        # each line keeps exactly its Gaussian mass over the union of its window's bins
        from scipy import special
        keep = r["keep"].astype(bool)
        nu, a = r["nu"][keep], r["alpha"][keep]
        lo_e = w.nu_min + (r["ilo"][keep] - 0.5) * w.dnu
        hi_e = w.nu_min + (r["ihi"][keep] + 0.5) * w.dnu
        cc = np.sqrt(np.log(2.0)) / a
        mass = 0.5 * (special.erf((hi_e - nu) * cc) - special.erf((lo_e - nu) * cc))
        assert (mass < 0.999).sum() > 10          # some windows are cut by the grid ends
        assert got.sum() * w.dnu == pytest.approx(np.sum(r["I"][keep] * mass), rel=1e-5)


@pytest.mark.parametrize("kind", ["binned_gauss_hwhm", "binned_voigt"])
def test_binned_every_tile(pxc, kind):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=1000, hwhm=0.03, threshold=0.0)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, kind)
    ref = H.oracle_run(c, kind=kind, threshold=0.0)["sigma"]
    for tile in range(pxc.NUM_TILES):
        ws.set_tile(pxc.PROFILES[kind], False, tile)
        sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
        assert ws.stats()["tile"] == tile
        H.check_sigma(H.sigma_phys(sig[0], e[0].item()), ref, f"{kind} tile {tile}")


def test_binned_backward_refused(pxc):
    import torch
    c = H.case("voigt_1e9", n_states=300_000, n_trans=1000, threshold=0.0)
    w = c["w"]
    ws = _ws(pxc, c)
    st, tr, prof, grid = H.device(c, "binned_voigt")
    wt = torch.zeros(w.n_grid, dtype=torch.float32, device="cuda")
    with pytest.raises(pxc.PxcError) as ei:
        pxc.pxc_cross_section_backward(ws, st, tr, (w.T, 0.0, w.P), grid, prof, wt)
    assert ei.value.code == 1
