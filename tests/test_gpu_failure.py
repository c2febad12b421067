"""Failure detection on the GPU without a fault: a bounded device wait that
runs out (on an mbarrier phase nothing completes, or on a shared-memory counter
nothing advances: the two kinds of wait the kernels use) ends its kernel within
a bounded time with SMPPI_DEV_TIMEOUT in the status word, and the context stays
usable: a Shield-MPPI update right after it returns the same status and matches the same
update on a fresh handle bit for bit.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _shield_update(S, pr):
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    S.smppi_shield_update(ctl.h, x0, V, Vs, 0, 0, 10)
    st, _ = ctl.sync_status()
    out = (x0.cpu().numpy(), V.cpu().numpy(), Vs.cpu().numpy())
    ctl.close()
    return st, out


@pytest.mark.parametrize("which", [0, 1])
def test_wait_runs_out_and_reports(S, which):
    pr = I.single_step_small()
    st0, ref = _shield_update(S, pr)
    assert st0 in (S.OK, S.ERR_STALLED)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.smppi_debug_wait_timeout(which, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    bits = int(status.item())
    print("wait %d gave up after %.3f s, status bits %d" % (which, dt, bits))
    assert bits == S.DEV_TIMEOUT
    assert 0.05 < dt < 5.0
    st1, out = _shield_update(S, pr)
    assert st1 == st0
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)


def test_wait_timeout_arguments(S):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SmppiError):
        S.smppi_debug_wait_timeout(2, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
