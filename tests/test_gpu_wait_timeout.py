"""Failure detection on the GPU without a fault: the profile kernel's waits for staged line
records are bounded.  With the bound set to 0 they give up at once; the call must come back with
PXC_ERR_TIMEOUT from the status check (not a hang, not a fault), and the same workspace must
then give the oracle's sigma again with the default bound."""
import pytest

from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pxc():
    import torch  # noqa: F401
    import paper_2609_17273_b300 as m
    m.load()
    return m


def test_wait_timeout_is_reported_and_the_workspace_recovers(pxc):
    c = H.case("voigt_1e9", n_states=300_000, n_trans=40_000, threshold=0.0)
    w = c["w"]
    ws = pxc.Workspace(max_states=len(c["E"]), max_lines=len(c["up"]), max_grid=w.n_grid)
    st, tr, prof, grid = H.device(c)
    ws.set_wait_limit(0)
    pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
    with pytest.raises(pxc.PxcError) as ei:
        ws.sync()
    assert ei.value.code == 5                     # PXC_ERR_TIMEOUT, latched and then cleared
    ws.sync()                                     # nothing latched any more
    ws.set_wait_limit()
    for _ in range(2):
        sig, e = pxc.pxc_cross_section(ws, st, tr, (w.T, 0.0, w.P), grid, prof, 0.0)
        ws.sync()
    r = H.oracle_run(c, threshold=0.0)
    H.check_sigma(H.sigma_phys(sig[0], e[0].item()), r["sigma"], "after a timeout")
    with pytest.raises(pxc.PxcError) as ei:
        ws.set_wait_limit(-1)
    assert ei.value.code == 1
