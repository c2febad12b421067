"""smppi_step_noalloc: the MPPI iteration for callers that cannot allocate device
memory (control loops that forbid allocation once running, runtimes that own
every device allocation).  It keeps its scratch in a fixed array inside the
library instead of a handle's workspace.

Checked against the handle-based smppi_step on the same inputs, two calls in a
row (the second starts from the first's V+, with the next iteration counter).
Both run the same kernels with the same launch shapes on the same inputs, so
costs and V+ must be bit-identical: a difference would mean that the fixed
scratch layout overlaps or keeps stale data.  Sizes beyond the limit are
refused with an argument error, and the documented limit of its error
reporting holds: a NaN start state still returns SMPPI_OK (the device status
word is not read back) and V+ lies on the lower corner of the control box.
Runs alone or after the other tests.
"""
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


@pytest.mark.parametrize("K,T", [(4096, 64), (1000, 51)])
def test_noalloc_matches_step_two_calls(S, K, T):
    pr = I.single_problem(K=K, T=T)
    ctl = S.Controller(pr.params, pr.track)        # existing entry point (handle workspace)
    x0 = ctl.tensor(pr.x0)
    V_ref = ctl.tensor(pr.V)
    V_na = ctl.tensor(pr.V)
    p = S.params_from_dict(pr.params, ctl.track)    # same parameters, no handle
    for it in range(2):
        S_ref = torch.empty(K, device="cuda")
        S_na = torch.empty(K, device="cuda")
        S.smppi_step(ctl.h, x0, V_ref, it, 0, S_ref, None)
        S.smppi_step_noalloc(p, x0, V_na, it, 0, S_na)
        torch.cuda.synchronize()
        assert ctl.sync_status()[0] == S.OK
        assert torch.equal(S_na, S_ref), it
        assert torch.equal(V_na, V_ref), it
    # without S_out the costs stay in the library's scratch; V+ is the same
    V_na2 = ctl.tensor(pr.V)
    S.smppi_step_noalloc(p, x0, V_na2, 0, 0, None)
    V_ref2 = ctl.tensor(pr.V)
    S.smppi_step(ctl.h, x0, V_ref2, 0, 0, None, None)
    torch.cuda.synchronize()
    assert torch.equal(V_na2, V_ref2)
    ctl.close()


def test_noalloc_nan_state_not_reported(S):
    pr = I.single_problem(K=1024, T=32)
    track = torch.as_tensor(pr.track, device="cuda")
    p = S.params_from_dict(pr.params, track)
    x0 = torch.as_tensor(pr.x0, device="cuda")
    x0[3] = float("nan")
    V = torch.as_tensor(pr.V, device="cuda")
    S.smppi_step_noalloc(p, x0, V, 0, 0)        # no exception: SMPPI_OK
    torch.cuda.synchronize()
    lo = torch.tensor([pr.params["u_min"][0], pr.params["u_min"][1]], device="cuda")
    assert torch.equal(V, lo.expand_as(V).contiguous())
    # the next call on clean inputs is unaffected
    x1 = torch.as_tensor(pr.x0, device="cuda")
    V1 = torch.as_tensor(pr.V, device="cuda")
    S.smppi_step_noalloc(p, x1, V1, 0, 0)
    ctl = S.Controller(pr.params, pr.track)
    V2 = ctl.tensor(pr.V)
    S.smppi_step(ctl.h, ctl.tensor(pr.x0), V2, 0, 0, None, None)
    torch.cuda.synchronize()
    assert torch.equal(V1, V2)
    ctl.close()


def test_noalloc_rejects_sizes_beyond_limit(S):
    pr = I.single_problem(K=65537, T=20)
    track = torch.as_tensor(pr.track, device="cuda")
    p = S.params_from_dict(pr.params, track)
    x0 = torch.as_tensor(pr.x0, device="cuda")
    V = torch.as_tensor(pr.V, device="cuda")
    with pytest.raises(S.SmppiError) as err:
        S.smppi_step_noalloc(p, x0, V, 0, 0)
    assert err.value.status == S.ERR_ARG
    assert "65536" in S.smppi_last_error(None)
