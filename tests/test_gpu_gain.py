"""GPU parity on two-temperature lists with inverted populations (gain, I < 0).

With T_vib > T_rot a line whose upper state has more vibrational but less rotational energy
than its lower state can have the larger population per degeneracy in its upper state; its
absorption intensity is then negative (Secs. 3.2-3.3, reading R10: such lines are kept when
|I| >= S_min, and the list exponent follows |I|).  The fixture is a seeded diatomic-like list in
which many lines are inverted and of the same magnitude as the normal ones.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu

TV, TR = 6000.0, 300.0


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


def _gain_case(seed=7, n_trans=40_000):
    rng = np.random.default_rng(seed)
    nv, nJ = 5, 80
    v = np.repeat(np.arange(nv), nJ)
    J = np.tile(np.arange(nJ), nv)
    Ev = 2000.0 * v
    # a seeded perturbation of every rotational energy keeps the Treanor exponent of every line
    # clear of exact zeros (where both sides would round an exactly cancelling difference)
    E = Ev + 10.0 * J * (J + 1.0) * (1.0 + rng.uniform(-0.02, 0.02, v.size))
    g = (2 * J + 1).astype(np.int32)
    lo = rng.integers(0, nv * nJ, n_trans)
    dv = rng.integers(1, 3, n_trans)
    dJ = rng.choice([-1, 0, 1], n_trans)
    vu = np.minimum(v[lo] + dv, nv - 1)
    Ju = np.clip(J[lo] + dJ, 0, nJ - 1)
    up = (vu * nJ + Ju).astype(np.int32)
    A = 10.0 ** rng.uniform(-2.0, 2.0, n_trans)
    w = H.synth.workload("doppler_1e5").scaled(n_states=E.size, n_trans=n_trans, nu_min=0.0, dnu=0.01,
                                                n_grid=1_200_001, cutoff=5.0, T=TR, T_vib=TV, P=1.0,
                                                profile="voigt", threshold=0.0)
    return {"w": w, "E": E, "g": g, "Ev": Ev, "up": up, "lo": lo.astype(np.int32), "A": A,
            "gr": rng.uniform(0.03, 0.1, n_trans).astype(np.float32),
            "ne": rng.uniform(0.4, 0.8, n_trans).astype(np.float32)}


def _sigma_abs(c, r):
    """The oracle's sum of |I_l| f_l: the scale of a signed sigma at each bin."""
    w = c["w"]
    return oracle.cross_section("voigt", r["nu"], np.abs(r["I"]), r["alpha"], r["gamma"], r["keep"], r["ilo"],
                                r["ihi"], w.nu_min, w.dnu, w.n_grid)


def _check_signed(got, ref, ref_abs, what):
    """The sigma criteria with the magnitude sum sum |I_l| f_l as the scale: a signed sigma passes
    through zero where absorption and gain cancel, and its rounding error there follows the
    magnitudes of the cancelling terms (as for the gradients' scale): max |d| <= 1e-4 of the peak
    magnitude, and |d| <= 1e-3 of the local magnitude sum wherever that is above 1e-6 of its peak."""
    m = ref_abs.max()
    d = np.abs(got - ref)
    assert d.max() <= H.SIG_ABS * m, f"{what}: max |d| / peak = {d.max() / m:.3e}"
    big = ref_abs > H.SIG_FLOOR * m
    rel = d[big] / ref_abs[big]
    assert rel.max() <= H.SIG_REL, f"{what}: worst per-bin rel = {rel.max():.3e}"


def _ws(pxc, c, n_c=1):
    return pxc.Workspace(max_states=len(c["E"]), max_lines=len(c["up"]), max_grid=c["w"].n_grid,
                         max_conditions=n_c)


def test_inverted_lines_intensities_and_threshold(pxc):
    c = _gain_case()
    w = c["w"]
    r0 = H.oracle_run(c, with_sigma=False, threshold=0.0)
    k0 = r0["keep"].astype(bool)
    neg = k0 & (r0["I"] < 0)
    assert neg.sum() > 1000 and (k0 & (r0["I"] > 0)).sum() > 1000
    # a threshold inside the distribution of the inverted lines' magnitudes
    mags = np.sort(np.abs(r0["I"][neg]))
    j = mags.size // 2
    while mags[j + 1] <= mags[j] * (1 + 1e-6):
        j += 1
    thr = float(np.sqrt(mags[j] * mags[j + 1]))
    st, tr, _, grid = H.device(c)
    ws = _ws(pxc, c)
    for threshold in (0.0, thr):
        nu, Is, k, nk = pxc.pxc_line_intensities(ws, st, tr, (TR, TV, 1.0), grid, w.cutoff, threshold)
        ws.sync()
        r = H.oracle_run(c, with_sigma=False, threshold=threshold)
        keep = r["keep"].astype(bool)
        assert np.array_equal(nu.cpu().numpy().view(np.uint64), r["nu"].view(np.uint64))
        assert int(nk.item()) == int(keep.sum())
        assert int(k.item()) == r["k"]
        Ig, Io = Is.cpu().numpy(), r["I_s"]
        assert np.array_equal(Ig != 0, Io != 0)
        assert np.all(np.sign(Ig) == np.sign(Io))
        ulp = np.spacing(np.abs(Io).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(Ig.astype(np.float64) - Io.astype(np.float64)) <= ulp)
        assert (Io[keep] < 0).any()
        if threshold > 0:
            assert keep.sum() < k0.sum() and (np.abs(r["I"][keep]) >= threshold).all()


def test_inverted_lines_cross_section(pxc):
    c = _gain_case(seed=9)
    w = c["w"]
    st, tr, prof, grid = H.device(c)
    ws = _ws(pxc, c)
    sig, e = pxc.pxc_cross_section(ws, st, tr, (TR, TV, 1.0), grid, prof)
    ws.sync()
    r = H.oracle_run(c)
    got = H.sigma_phys(sig[0], e[0].item())
    assert r["sigma"].min() < -1e-4 * np.abs(r["sigma"]).max(), "fixture has regions of net gain"
    ref_abs = _sigma_abs(c, r)
    _check_signed(got, r["sigma"], ref_abs, "inverted populations")
    assert int(e[0].item()) == r["k"]
    # the same lines in a batched call next to an LTE condition (one sort, two intensity slots)
    ws2 = _ws(pxc, c, n_c=2)
    sig2, e2 = pxc.pxc_cross_section(ws2, st, tr, [(TR, TV, 1.0), (TR, 0.0, 1.0)], grid, prof)
    ws2.sync()
    _check_signed(H.sigma_phys(sig2[0], e2[0].item()), r["sigma"], ref_abs, "inverted, batched")
    r_lte = H.oracle_run(c, T_vib=0.0)
    assert r_lte["sigma"].min() >= 0.0
    H.check_sigma(H.sigma_phys(sig2[1], e2[1].item()), r_lte["sigma"], "LTE, batched")
