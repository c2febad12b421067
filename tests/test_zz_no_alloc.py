"""smppi_step_noalloc: the MPPI iteration for callers that cannot allocate device
memory (control loops that forbid allocation once running, runtimes that own
every device allocation).  It keeps its scratch in a fixed array inside the
library instead of a handle's workspace.

Checked against the handle-based smppi_step on the same inputs, two calls in a
row (the second starts from the first's V+, with the next iteration counter),
within the update tolerance of the other GPU tests; and sizes beyond its limit
are refused with an argument error.  Runs alone or after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402

V_TOL = 1e-5          # the control-update tolerance of the GPU parity tests
S_TOL = 1e-4          # relative, rollout costs


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
        sr, sn = S_ref.cpu().numpy(), S_na.cpu().numpy()
        assert np.all(np.abs(sn - sr) <= S_TOL * (np.abs(sr) + 1.0))
        assert np.max(np.abs(V_na.cpu().numpy() - V_ref.cpu().numpy())) <= V_TOL, it
    # without S_out the costs stay in the library's scratch; V+ is the same
    V_na2 = ctl.tensor(pr.V)
    S.smppi_step_noalloc(p, x0, V_na2, 0, 0, None)
    V_ref2 = ctl.tensor(pr.V)
    S.smppi_step(ctl.h, x0, V_ref2, 0, 0, None, None)
    torch.cuda.synchronize()
    assert np.max(np.abs(V_na2.cpu().numpy() - V_ref2.cpu().numpy())) <= V_TOL
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
