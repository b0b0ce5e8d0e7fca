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
