"""GPU adjoint (pxc_cross_section_backward and the autograd Function) against the FP64
oracle adjoint and against central finite differences of the GPU forward pass.

The GPU returns gradients of L_s = sum_i w_i sigma_s,i with sigma = sigma_s 2^k, i.e.
the physical gradients times 2^-k.  Per-line gradients are sums of w f over a window
with random-sign w, so they are compared relative to max(|g|, the same sum with |w|)
(the condition number of the sum): within 1e-3 per line, 1e-4 for the scalars.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu

LINE_TOL = 1e-3
SCALAR_TOL = 1e-4


@pytest.fixture(scope="module")
def pxc():
    import paper_2609_17273_b300 as m
    m.load()
    return m


def _setup(pxc, name, kind, n_trans, **kw):
    import torch
    c = H.case(name, n_trans=n_trans, **kw)
    w = c["w"]
    ws = pxc.Workspace(max_states=len(c["E"]), max_lines=n_trans, max_grid=w.n_grid)
    st, tr, prof, grid = H.device(c, kind)
    wts = w.weights()
    wt = torch.from_numpy(wts).cuda()
    return c, w, ws, st, tr, prof, grid, wts, wt


@pytest.mark.parametrize("name,kind,n", [("nlte_1e7", "voigt", 20_000), ("voigt_1e7", "voigt", 30_000),
                                         ("voigt_1e7", "lorentz", 30_000), ("doppler_1e5", "gauss_doppler", 30_000)])
def test_adjoint_matches_oracle(pxc, name, kind, n):
    c, w, ws, st, tr, prof, grid, wts, wt = _setup(pxc, name, kind, n)
    cond = (w.T, w.T_vib, w.P)
    sig, e = pxc.pxc_cross_section(ws, st, tr, cond, grid, prof)
    k = int(e[0].item())
    out = pxc.pxc_cross_section_backward(ws, st, tr, cond, grid, prof, wt)
    ws.sync()
    r = H.oracle_run(c, kind=kind, with_sigma=False)
    gd = oracle.cross_section_grad(kind, c["E"], c["Ev"], c["up"], c["lo"], c["A"], r["nu"], r["I"], r["alpha"],
                                   r["gamma"], c["ne"], r["keep"], r["ilo"], r["ihi"], w.T, w.T_vib, w.P, r["Q"],
                                   w.nu_min, w.dnu, wts.astype(np.float64))
    sc = 2.0 ** -k
    keep = r["keep"].astype(bool)
    A = c["A"].astype(np.float64)
    # dL/dA
    ref = gd["dA"] * sc
    scale = np.maximum(np.abs(ref), np.where(keep, r["I"] / A * gd["Gabs"][:, 0], 0.0) * sc)
    got = out["dA"].double().cpu().numpy()
    m = scale > 1e-6 * scale.max()
    assert np.all(np.abs(got - ref)[m] <= LINE_TOL * scale[m]), \
        f"dA worst {np.max(np.abs(got - ref)[m] / scale[m]):.2e}"
    assert np.all(np.abs(got[~m]) <= 1e-5 * scale.max())
    if kind in ("voigt", "lorentz"):
        fac = np.where(keep, r["gamma"] / np.maximum(c["gr"].astype(np.float64), 1e-30), 0.0)
        ref = gd["dgamma_ref"] * sc
        scale = np.maximum(np.abs(ref), r["I"] * fac * gd["Gabs"][:, 2] * sc)
        got = out["dgamma_ref"].double().cpu().numpy()
        m = scale > 1e-6 * scale.max()
        assert np.all(np.abs(got - ref)[m] <= LINE_TOL * scale[m]), \
            f"dgamma_ref worst {np.max(np.abs(got - ref)[m] / scale[m]):.2e}"
    for key, akey in (("dT", "dT_abs"), ("dTvib", "dTvib_abs"), ("dP", "dP_abs")):
        refv = gd[key] * sc
        sv = max(abs(refv), gd[akey] * sc)
        if sv == 0:
            continue
        assert abs(out[key].item() - refv) <= SCALAR_TOL * sv, f"{key}: {out[key].item()} vs {refv} (scale {sv})"


def test_adjoint_matches_finite_differences(pxc):
    import torch
    c, w, ws, st, tr, prof, grid, wts, wt = _setup(pxc, "nlte_1e7", "voigt", 20_000)

    def loss(T, Tv, P):
        s, e = pxc.pxc_cross_section(ws, st, tr, (T, Tv, P), grid, prof)
        return float(np.dot(wts.astype(np.float64), H.sigma_phys(s[0], e[0].item())))

    cond = (w.T, w.T_vib, w.P)
    s, e = pxc.pxc_cross_section(ws, st, tr, cond, grid, prof)
    k = int(e[0].item())
    out = pxc.pxc_cross_section_backward(ws, st, tr, cond, grid, prof, wt)
    g = {key: out[key].item() * 2.0 ** k for key in ("dT", "dTvib", "dP")}
    for key, i in (("dT", 0), ("dTvib", 1), ("dP", 2)):
        x0 = list(cond)
        fds = []
        for h in (1e-3, 5e-4):
            xp, xm = list(x0), list(x0)
            xp[i] *= 1 + h
            xm[i] *= 1 - h
            fds.append((loss(*xp) - loss(*xm)) / (2 * h * x0[i]))
        est = abs(fds[0] - fds[1]) + 1e-3 * abs(fds[1])
        assert abs(g[key] - fds[1]) <= 3 * est + 1e-12, f"{key}: adjoint {g[key]} vs FD {fds}"
    del torch


def test_autograd_function(pxc):
    import torch
    c, w, ws, st, tr, prof, grid, wts, wt = _setup(pxc, "nlte_1e7", "voigt", 10_000)
    T = torch.tensor(w.T, dtype=torch.float64, requires_grad=True)
    Tv = torch.tensor(w.T_vib, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(w.P, dtype=torch.float64, requires_grad=True)
    gref = prof.gamma_ref.clone().requires_grad_(True)
    A = tr.A.clone().requires_grad_(True)
    sig, e = pxc.CrossSection.apply(ws, st, tr.upper, tr.lower, grid, prof, 0.0, T, Tv, P, gref, A)
    L = (sig.double() * wt.double()).sum()
    L.backward()
    out = pxc.pxc_cross_section_backward(ws, st, tr, (w.T, w.T_vib, w.P), grid, prof, wt)
    assert T.grad.item() == pytest.approx(out["dT"].item(), rel=1e-12)
    assert Tv.grad.item() == pytest.approx(out["dTvib"].item(), rel=1e-12)
    assert P.grad.item() == pytest.approx(out["dP"].item(), rel=1e-12)
    assert torch.equal(A.grad.float(), out["dA"]) and torch.equal(gref.grad, out["dgamma_ref"])


def test_reuse_of_the_forward_line_list(pxc):
    """pxc_set_reuse_forward: a backward right after an identical forward reads the forward's sorted
    line list and returns bit-identical gradients to a backward that recomputes it; an intervening
    call with other arguments discards the list and the backward recomputes (same results again)."""
    import torch
    c, w, ws, st, tr, prof, grid, wts, wt = _setup(pxc, "nlte_1e7", "voigt", 20_000)
    cond = (w.T, w.T_vib, w.P)
    pxc.pxc_cross_section(ws, st, tr, cond, grid, prof)
    ref = pxc.pxc_cross_section_backward(ws, st, tr, cond, grid, prof, wt)
    ws.sync()
    ref = {k: v.clone() for k, v in ref.items()}
    ws.set_reuse_forward(True)
    pxc.pxc_cross_section(ws, st, tr, cond, grid, prof)
    got = pxc.pxc_cross_section_backward(ws, st, tr, cond, grid, prof, wt)
    ws.sync()
    for k in ref:
        assert torch.equal(got[k], ref[k]), k
    # a forward at another condition in between: the backward at the first condition recomputes
    pxc.pxc_cross_section(ws, st, tr, (w.T * 1.1, w.T_vib, w.P), grid, prof)
    again = pxc.pxc_cross_section_backward(ws, st, tr, cond, grid, prof, wt)
    ws.sync()
    for k in ref:
        assert torch.equal(again[k], ref[k]), k
    ws.set_reuse_forward(False)
