"""Shared helpers of the parity tests: seeded cases, device upload, tolerance checks."""
from __future__ import annotations

import numpy as np

import oracle
import synth

# sigma tolerances: max |d| <= 1e-4 * max(sigma_ref), and per bin |d|/sigma_ref <= 1e-3
# wherever sigma_ref > 1e-6 * max(sigma_ref)
SIG_ABS = 1e-4
SIG_REL = 1e-3
SIG_FLOOR = 1e-6


def case(name: str, n_trans: int | None = None, n_states: int | None = None, **kw):
    """Seeded synthetic case from a named workload, optionally scaled down."""
    w = synth.workload(name)
    upd = dict(kw)
    if n_trans is not None:
        upd["n_trans"] = n_trans
    if n_states is not None:
        upd["n_states"] = n_states
    w = w.scaled(**upd) if upd else w
    E, g, Ev = w.states()
    up, lo, A = w.transitions()
    gr, ne = w.broadening()
    return {"w": w, "E": E, "g": g, "Ev": Ev, "up": up, "lo": lo, "A": A, "gr": gr, "ne": ne}


def oracle_run(c, kind=None, T=None, T_vib=None, P=None, threshold=None, with_sigma=True, literal=False,
               emission=False, n_vib=None):
    w = c["w"]
    return oracle.run(c["E"], c["g"], c["Ev"], c["up"], c["lo"], c["A"], c["gr"], c["ne"],
                      kind=kind or w.profile, T=w.T if T is None else T,
                      T_vib=w.T_vib if T_vib is None else T_vib, P=w.P if P is None else P,
                      mass_da=w.mass_da, hwhm=w.hwhm, nu_min=w.nu_min, dnu=w.dnu, n_grid=w.n_grid,
                      cut=w.cutoff, threshold=w.threshold if threshold is None else threshold,
                      with_sigma=with_sigma, emission=emission, n_vib=n_vib)


def device(c, kind=None):
    import torch
    import paper_2609_17273_b300 as pxc
    w = c["w"]
    st = pxc.States(torch.from_numpy(c["E"]).cuda(), torch.from_numpy(c["g"]).cuda(),
                    torch.from_numpy(c["Ev"]).cuda())
    tr = pxc.Transitions(torch.from_numpy(c["up"]).cuda(), torch.from_numpy(c["lo"]).cuda(),
                         torch.from_numpy(c["A"]).cuda())
    prof = pxc.Profile(kind or w.profile, w.cutoff, w.mass_da, w.hwhm,
                       torch.from_numpy(c["gr"]).cuda(), torch.from_numpy(c["ne"]).cuda(), 296.0)
    grid = (w.nu_min, w.dnu, w.n_grid)
    return st, tr, prof, grid


def sigma_phys(sig, e):
    """FP32 scaled sigma and its exponent -> float64 physical values."""
    return np.ldexp(sig.double().cpu().numpy(), int(e))


def check_sigma(got, ref, what=""):
    m = np.abs(ref).max()
    assert m > 0, f"{what}: reference is identically zero"
    d = np.abs(got - ref)
    assert d.max() <= SIG_ABS * m, f"{what}: max |d| / max = {d.max() / m:.3e}"
    big = np.abs(ref) > SIG_FLOOR * m
    rel = d[big] / np.abs(ref[big])
    assert rel.max() <= SIG_REL, f"{what}: worst per-bin rel = {rel.max():.3e} at {np.nonzero(big)[0][rel.argmax()]}"
    return {"max_abs_rel": float(d.max() / m), "worst_bin_rel": float(rel.max()),
            "l1": float(d.sum() / np.abs(ref).sum())}
