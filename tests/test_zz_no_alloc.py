"""The no-allocation partition function against the workspace one.

pxc_partition_function_noalloc serves callers that may not allocate device
memory; it keeps its scratch in a fixed array inside the library.  This file is
collected last so that, if it fails, a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    import torch
    import paper_2609_17273_b300 as pxc
    pxc.load()
    c = H.case("nlte_1e7", n_trans=10)
    st, _, _, _ = H.device(c)
    ws = pxc.Workspace(max_states=len(c["E"]), max_lines=16, max_grid=16, max_conditions=8)
    calls = [[(296.0, 0.0, 1.0), (1500.0, 0.0, 1.0), (1200.0, 2500.0, 1.0)],
             [(3000.0, 0.0, 1.0), (800.0, 1600.0, 1.0)]]
    for conds in calls:
        Qa, dQa, status = pxc.pxc_partition_function_noalloc(st, conds)
        Qb, dQb = pxc.pxc_partition_function(ws, st, conds)
        ws.sync()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        a, b = Qa.cpu().numpy(), Qb.cpu().numpy()
        assert np.allclose(a, b, rtol=1e-12, atol=0)
        assert np.allclose(dQa.cpu().numpy(), dQb.cpu().numpy(), rtol=1e-10, atol=0)
    # beyond the stated maximum: a clear error, nothing launched
    with pytest.raises(pxc.PxcError) as e:
        pxc.pxc_partition_function_noalloc(st, [(500.0, 0.0, 1.0)] * 65)
    assert e.value.code == 7


def test_noalloc_vibronic_densities_and_device_statuses():
    import torch
    import paper_2609_17273_b300 as pxc
    pxc.load()
    c = H.case("nlte_1e7", n_trans=10)
    w = c["w"]
    st, _, _, _ = H.device(c)
    ws = pxc.Workspace(max_states=len(c["E"]), max_lines=16, max_grid=16, max_conditions=4)
    # vibronic-density populations (T is T_rot, no T_vib)
    nv = torch.from_numpy(w.vib_densities()).cuda()
    std = pxc.States(st.E, st.g, st.E_vib, nv)
    conds = [(1200.0, 0.0, 1.0), (700.0, 0.0, 1.0)]
    Qa, dQa, status = pxc.pxc_partition_function_noalloc(std, conds)
    Qb, dQb = pxc.pxc_partition_function(ws, std, conds)
    ws.sync()
    assert int(status.item()) == 0
    assert np.allclose(Qa.cpu().numpy(), Qb.cpu().numpy(), rtol=1e-12, atol=0)
    assert np.allclose(dQa.cpu().numpy(), dQb.cpu().numpy(), rtol=1e-10, atol=0)
    # the unclamped level law: energies far below zero overflow the Boltzmann factor
    d = H.synth.workload("doppler_1e5")
    El, gl, _ = d.states(literal=True)
    stl = pxc.States(torch.from_numpy(El).cuda(), torch.from_numpy(gl).cuda(), None)
    _, _, status = pxc.pxc_partition_function_noalloc(stl, [(d.T, 0.0, 1.0)])
    assert int(status.item()) == 4  # PXC_ERR_OVERFLOW
    # an infinite energy
    Ei = c["E"].copy()
    Ei[123] = np.inf
    sti = pxc.States(torch.from_numpy(Ei).cuda(), st.g, None)
    _, _, status = pxc.pxc_partition_function_noalloc(sti, [(1500.0, 0.0, 1.0)])
    assert int(status.item()) == 3  # PXC_ERR_NONFINITE
    # the shared error word is cleared at the start of every call: a valid call after the bad
    # ones reports OK and the workspace entry point's Q
    Qa, _, status = pxc.pxc_partition_function_noalloc(st, [(1500.0, 0.0, 1.0)])
    Qb, _ = pxc.pxc_partition_function(ws, st, [(1500.0, 0.0, 1.0)])
    ws.sync()
    assert int(status.item()) == 0
    assert Qa.item() == pytest.approx(Qb.item(), rel=1e-12)
