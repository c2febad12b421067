"""Start states without a nearest centreline segment (a position that is NaN,
infinite or beyond ~1e19 m).  The nearest-segment search then starts from
segment 0 and sets the NUMERIC bit of the status word (smppi.h), so every table
access stays in bounds; the handle, and every other problem of a batch, is
unaffected.  The position is planted from the host into the device state.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402

BAD = [("X", 3, float("nan")), ("Y", 4, float("inf")), ("X", 3, 3.0e19)]


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


@pytest.mark.parametrize("name,j,val", BAD)
def test_step_and_shield_report_numeric(S, name, j, val):
    pr = I.single_step_small()
    ctl = S.Controller(pr.params, pr.track, max_seq=4)
    x0 = ctl.tensor(pr.x0)
    x0[j] = val
    V = ctl.tensor(pr.V)
    ctl.step(x0, V)
    st, bits = ctl.sync_status()
    assert st == S.ERR_NUMERIC and bits & S.DEV_NUMERIC
    lo = np.array([pr.params["u_min"][0], pr.params["u_min"][1]], np.float32)
    assert np.array_equal(V.cpu().numpy(), np.broadcast_to(lo, V.shape))   # NaN costs: lower corner
    # whole update (rollouts, update, shield tail, closed-loop step)
    x0 = ctl.tensor(pr.x0)
    x0[j] = val
    V, Vs = ctl.tensor(pr.V), ctl.tensor(pr.V)
    S.smppi_shield_update(ctl.h, x0, V, Vs, 0, 0, 10)
    st, bits = ctl.sync_status()
    assert bits & S.DEV_NUMERIC
    # the repair on its own: block repair (mode 1) and BFGS (mode 2) searches
    xs = ctl.tensor(np.repeat(pr.x0[None], 4, 0))
    xs[1, j] = val
    Vin = ctl.tensor(np.zeros((4, pr.params["T"], 2), np.float32))
    Vout = torch.empty_like(Vin)
    for mode in (1, 2):
        S.smppi_repair(ctl.h, 4, xs, Vin, Vout, 5, mode)
        st, bits = ctl.sync_status()
        assert bits & S.DEV_NUMERIC, mode
    # host buffers: refused before anything is enqueued
    hx = pr.x0.copy()
    hx[j] = val
    hV, hVs = pr.V.copy(), pr.V.copy()
    with pytest.raises(S.SmppiError) as err:
        S.smppi_shield_update(ctl.h, hx.ctypes.data, hV.ctypes.data, hVs.ctypes.data, 0, 0, 10,
                              None, True)
    assert err.value.status == S.ERR_ARG
    # the handle stays usable
    ctl.step(ctl.tensor(pr.x0), ctl.tensor(pr.V))
    assert ctl.sync_status()[0] == S.OK
    ctl.close()


def test_batch_other_problems_unaffected(S):
    ib = I.uneven_instances(n_inst=4, seed=3, K_lo=200, K_hi=600, T_lo=20, T_hi=40)
    outs = []
    for plant in (False, True):
        bt = S.Batch(ib, block_rollouts=128)
        if plant:
            bt.x0[2, 3] = float("nan")
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, 0, 5)
        st, bits = S.smppi_batch_sync_status(bt.b)
        assert bool(bits & S.DEV_NUMERIC) == plant, bits
        outs.append((bt.x0.cpu().numpy(), bt.split(bt.V), bt.split(bt.V_safe)))
        bt.close()
    (x_a, V_a, Vs_a), (x_b, V_b, Vs_b) = outs
    for i in (0, 1, 3):
        assert np.array_equal(x_a[i], x_b[i])
        assert np.array_equal(V_a[i], V_b[i]) and np.array_equal(Vs_a[i], Vs_b[i])
