"""GPU parity of emission intensities and cross sections, vibronic-density populations and
the cooling function against the FP64 oracle (same seeded inputs, same tolerances as the
absorption path: nu and the kept set bit-exact, I_s within 1 FP32 ulp, sigma within 1e-4
of its peak and 1e-3 per bin)."""
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


def _states(pxc, c, nv=None):
    import torch
    return pxc.States(torch.from_numpy(c["E"]).cuda(), torch.from_numpy(c["g"]).cuda(),
                      torch.from_numpy(c["Ev"]).cuda(), None if nv is None else torch.from_numpy(nv).cuda())


def _check_lines(pxc, ws, c, st, tr, cond, r):
    w = c["w"]
    nu, Is, k, nk = pxc.pxc_line_intensities(ws, st, tr, cond, (w.nu_min, w.dnu, w.n_grid), w.cutoff, w.threshold)
    ws.sync()
    assert np.array_equal(nu.cpu().numpy().view(np.uint64), r["nu"].view(np.uint64))
    assert int(nk.item()) == int(r["keep"].sum())
    assert int(k.item()) == r["k"]
    Ig, Io = Is.cpu().numpy().astype(np.float64), r["I_s"].astype(np.float64)
    ulp = np.spacing(np.abs(r["I_s"]).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(Ig - Io) <= ulp)


@pytest.mark.parametrize("name,kw", [("doppler_1e5", {}),
                                     ("voigt_1e9", dict(n_states=400_000, n_trans=300_000))])
def test_emission_line_intensities_bit_exact(pxc, name, kw):
    c = H.case(name, **kw)
    w = c["w"]
    ws = _ws(pxc, c)
    ws.set_emission(True)
    st, tr, _, _ = H.device(c)
    r = H.oracle_run(c, with_sigma=False, emission=True)
    assert r["keep"].sum() > 1000
    _check_lines(pxc, ws, c, st, tr, (w.T, w.T_vib, w.P), r)


def test_emission_cross_section_polyatomic_with_threshold(pxc):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=60_000, threshold=1e-35)
    w = c["w"]
    ws = _ws(pxc, c)
    ws.set_emission(True)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, w.threshold)
    s = ws.stats()
    r = H.oracle_run(c, emission=True)
    r0 = H.oracle_run(c, emission=True, threshold=0.0, with_sigma=False)
    band = r0["keep"].astype(bool) & (np.abs(np.abs(r0["I"]) / w.threshold - 1.0) < 1e-9)
    assert not band.any(), "fixture has lines within the threshold rounding band"
    assert s["n_kept"] == int(r["keep"].sum()) and 0 < s["n_kept"] < int(r0["keep"].sum())
    assert int(e[0].item()) == r["k"]
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "emission")


def test_emission_two_temperature_cross_section(pxc):
    c = H.case("nlte_1e7", n_trans=150_000)
    w = c["w"]
    ws = _ws(pxc, c)
    ws.set_emission(True)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, w.T_vib, w.P), grid, prof)
    r = H.oracle_run(c, emission=True)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "emission 2T")


# --------------------------------------------------------------------------- vibronic densities

def _density_case(n_trans=150_000):
    c = H.case("nlte_1e7", n_trans=n_trans)
    return c, c["w"].vib_densities()


def test_density_partition_function(pxc):
    c, nv = _density_case(1000)
    ws = _ws(pxc, c, n_c=3)
    st = _states(pxc, c, nv)
    conds = [(300.0, 0.0, 1.0), (1200.0, 0.0, 1.0), (4000.0, 0.0, 1.0)]
    Q, dQ = pxc.pxc_partition_function(ws, st, conds)
    ws.sync()
    for i, (T, _, _) in enumerate(conds):
        ref = oracle.partition_density(c["E"], c["g"], c["Ev"], nv, T)
        assert Q[i].item() == pytest.approx(ref[0], rel=1e-12)
        assert dQ[i, 0].item() == pytest.approx(ref[1], rel=1e-10)
        assert dQ[i, 1].item() == 0.0


@pytest.mark.parametrize("emission", [False, True])
def test_density_line_intensities_bit_exact(pxc, emission):
    c, nv = _density_case(200_000)
    w = c["w"]
    ws = _ws(pxc, c)
    ws.set_emission(emission)
    st = _states(pxc, c, nv)
    _, tr, _, _ = H.device(c)
    r = H.oracle_run(c, T_vib=0.0, with_sigma=False, emission=emission, n_vib=nv)
    assert r["keep"].sum() > 1000
    _check_lines(pxc, ws, c, st, tr, (w.T, 0.0, w.P), r)


@pytest.mark.parametrize("emission", [False, True])
def test_density_cross_section(pxc, emission):
    c, nv = _density_case()
    w = c["w"]
    ws = _ws(pxc, c)
    ws.set_emission(emission)
    st = _states(pxc, c, nv)
    _, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof)
    r = H.oracle_run(c, T_vib=0.0, emission=emission, n_vib=nv)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], f"density emission={emission}")


def test_batched_emission_table_matches_oracle(pxc):
    c = H.case("voigt_1e9", n_states=200_000, n_trans=20_000, threshold=0.0)
    conds = [(T, 0.0, P) for T in (300.0, 3000.0) for P in (1e-3, 1.0)]
    ws = _ws(pxc, c, n_c=len(conds), n_temps=2)
    ws.set_emission(True)
    st, tr, prof, grid = H.device(c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, conds, grid, prof)
    for i, (T, _, P) in enumerate(conds):
        r = H.oracle_run(c, T=T, P=P, threshold=0.0, emission=True)
        H.check_sigma(H.sigma_phys(sig[i], e[i].item()), r["sigma"], f"batched emission T={T} P={P}")


# --------------------------------------------------------------------------- cooling function

@pytest.mark.parametrize("model", ["lte", "2T", "density"])
def test_cooling_function_matches_oracle(pxc, model):
    c, nv = _density_case(500_000)
    ws = _ws(pxc, c, n_c=4)
    if model == "lte":
        conds, st, dens = [(T, 0.0, 1.0) for T in (300.0, 1000.0, 3000.0, 8000.0)], _states(pxc, c), None
    elif model == "2T":
        conds, st, dens = [(T, 2500.0, 1.0) for T in (300.0, 1200.0)], _states(pxc, c), None
    else:
        conds, st, dens = [(T, 0.0, 1.0) for T in (500.0, 1200.0, 4000.0)], _states(pxc, c, nv), nv
    _, tr, _, _ = H.device(c)
    W, Q = pxc.pxc_cooling_function(ws, st, tr, conds)
    ws.sync()
    for i, (T, Tv, _) in enumerate(conds):
        if dens is not None:
            Qr = oracle.partition_density(c["E"], c["g"], c["Ev"], dens, T)[0]
        else:
            Qr = oracle.partition(c["E"], c["g"], c["Ev"] if Tv > 0 else None, T, Tv)[0]
        Wr = oracle.cooling_function(c["E"], c["g"], c["Ev"], c["up"], c["lo"], c["A"], T, Tv, Qr, n_vib=dens)
        assert Q[i].item() == pytest.approx(Qr, rel=1e-12)
        assert W[i].item() == pytest.approx(Wr, rel=1e-11), (model, T)


def test_cooling_function_polyatomic_f32_A(pxc):
    c = H.case("voigt_1e9", n_states=400_000, n_trans=1_000_000)
    ws = _ws(pxc, c, n_c=2)
    st, tr, _, _ = H.device(c)
    W, _ = pxc.pxc_cooling_function(ws, st, tr, [(1000.0, 0.0, 1.0), (2000.0, 0.0, 1.0)])
    ws.sync()
    for i, T in enumerate((1000.0, 2000.0)):
        Qr = oracle.partition(c["E"], c["g"], None, T)[0]
        Wr = oracle.cooling_function(c["E"], c["g"], None, c["up"], c["lo"], c["A"], T, 0.0, Qr)
        assert W[i].item() == pytest.approx(Wr, rel=1e-11)


def test_emission_and_density_argument_errors(pxc):
    c, nv = _density_case(1000)
    w = c["w"]
    ws = _ws(pxc, c)
    _, tr, prof, grid = H.device(c)
    import torch
    st_bad = pxc.States(torch.from_numpy(c["E"]).cuda(), torch.from_numpy(c["g"]).cuda(), None,
                        torch.from_numpy(nv).cuda())
    with pytest.raises(pxc.PxcError) as ei:       # densities need E_vib
        pxc.pxc_partition_function(ws, st_bad, [(500.0, 0.0, 1.0)])
    assert ei.value.code == 1
    st = _states(pxc, c, nv)
    with pytest.raises(pxc.PxcError) as ei:       # densities with T_vib > 0 are ambiguous
        pxc.pxc_cross_section(ws, st, tr, (500.0, 900.0, 1.0), grid, prof)
    assert ei.value.code == 1
    wt = torch.zeros(w.n_grid, dtype=torch.float32, device="cuda")
    with pytest.raises(pxc.PxcError):             # the adjoint is absorption with LTE / 2T only
        pxc.pxc_cross_section_backward(ws, st, tr, (500.0, 0.0, 1.0), grid, prof, wt)
    ws.set_emission(True)
    with pytest.raises(pxc.PxcError):
        pxc.pxc_cross_section_backward(ws, _states(pxc, c), tr, (500.0, 0.0, 1.0), grid, prof, wt)
    ws.set_emission(False)
    ws.sync()
