"""CUDA-graph capture and replay of pxc_cross_section (pxc_set_graphs).

A replayed call must give exactly the bits of the direct call on the same data, follow changes
of the device data behind the same pointers, capture again for a different call, and leave
accumulate mode uncaptured; the batched table it replays still matches the oracle.
"""
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


def test_graph_replay_is_bit_identical_and_follows_the_data(pxc):
    import torch
    c = H.case("voigt_1e9", n_states=200_000, n_trans=30_000, threshold=0.0)
    w = c["w"]
    conds = [(T, 0.0, P) for T in (500.0, 2000.0) for P in (1e-3, 0.1, 10.0)]
    st, tr, prof, grid = H.device(c)
    wsd = H_ws = pxc.Workspace(max_states=len(c["E"]), max_lines=len(c["up"]), max_grid=w.n_grid,
                               max_conditions=len(conds), max_temperatures=2)
    wsg = pxc.Workspace(max_states=len(c["E"]), max_lines=len(c["up"]), max_grid=w.n_grid,
                        max_conditions=len(conds), max_temperatures=2)
    wsg.set_graphs(True)
    a, ea = pxc.pxc_cross_section(wsd, st, tr, conds, grid, prof)
    sig = torch.empty_like(a)
    se = torch.empty_like(ea)
    pxc.pxc_cross_section(wsg, st, tr, conds, grid, prof, sigma=sig, sigma_exp=se)   # capture + launch
    wsg.sync()
    assert torch.equal(sig, a) and torch.equal(se, ea)
    sig.zero_()
    n0 = pxc.kernel_launches()
    pxc.pxc_cross_section(wsg, st, tr, conds, grid, prof, sigma=sig, sigma_exp=se)   # replay
    wsg.sync()
    assert pxc.kernel_launches() - n0 > 20  # the replay counts the graph's kernels
    assert torch.equal(sig, a) and torch.equal(se, ea)
    assert wsg.graph_stats() == {"captures": 1, "replays": 1, "cached": 1}
    s_d, s_g = wsd.stats(), wsg.stats()
    assert s_d == s_g
    # new values behind the same pointers: the replay reads them
    tr.A.mul_(torch.linspace(0.5, 3.0, tr.A.numel(), dtype=tr.A.dtype, device=tr.A.device))
    prof.gamma_ref.mul_(1.7)
    a2, ea2 = pxc.pxc_cross_section(wsd, st, tr, conds, grid, prof)
    pxc.pxc_cross_section(wsg, st, tr, conds, grid, prof, sigma=sig, sigma_exp=se)
    wsg.sync()
    assert not torch.equal(a2, a)
    assert torch.equal(sig, a2) and torch.equal(se, ea2)
    assert wsg.graph_stats()["replays"] == 2
    # the replayed table against the oracle at two of its conditions
    c2 = dict(c)
    c2["A"] = tr.A.cpu().numpy()
    c2["gr"] = prof.gamma_ref.cpu().numpy()
    for j in (0, len(conds) - 1):
        T, _, P = conds[j]
        r = H.oracle_run(c2, T=T, P=P, threshold=0.0)
        H.check_sigma(H.sigma_phys(sig[j], se[j].item()), r["sigma"], f"graph replay T={T} P={P}")
    # a different call is a new capture; the single-condition path is captured as well
    b, eb = pxc.pxc_cross_section(wsg, st, tr, conds[:1] * 1 + conds[1:2], grid, prof)
    one = pxc.pxc_cross_section(wsg, st, tr, conds[2], grid, prof)
    wsg.sync()
    assert wsg.graph_stats()["captures"] == 3
    ref_one = pxc.pxc_cross_section(wsd, st, tr, conds[2], grid, prof)
    wsd.sync()
    assert torch.equal(one[0], ref_one[0]) and torch.equal(one[1], ref_one[1])
    # accumulate mode is never captured
    wsg.set_accumulate(True)
    s1 = torch.zeros(1, w.n_grid, dtype=torch.float32, device="cuda")
    e1 = torch.full((1,), pxc.PXC_EXP_EMPTY, dtype=torch.int32, device="cuda")
    pxc.pxc_cross_section(wsg, st, tr, conds[2], grid, prof, sigma=s1, sigma_exp=e1)
    wsg.set_accumulate(False)
    wsg.sync()
    assert wsg.graph_stats()["captures"] == 3
    assert torch.equal(s1, ref_one[0]) and torch.equal(e1, ref_one[1])
    wsg.set_graphs(False)
    assert wsg.graph_stats()["cached"] == 0
    del torch, H_ws
