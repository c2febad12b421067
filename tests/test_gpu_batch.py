"""Batched persistent Shield-MPPI (smppi_batch_*) against the FP64 oracle.

Problems with uneven K, T, tracks and half-widths run in one launch.  At every
closed-loop step the device arrays are set to the ORACLE's state (oracle ->
GPU only), one batch update runs, and every problem's outputs are compared
with the oracle's own update of that state: the warm-started V (shift of V+)
within the update tolerance bound, V_safe within 1e-4 (unless a line-search
decision differs: a flip), the next state within 1e-4 relative.  Graph
replays equal plain steps bit for bit; the autotuner picks a legal shape.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import V_REP, X_REL, rel_err, update_bound  # noqa: E402


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


@pytest.fixture(scope="module")
def ib():
    return I.uneven_instances(n_inst=12, seed=5, K_lo=64, K_hi=2048, T_lo=20, T_hi=80)


def _set_state(bt, xs, Vs):
    bt.x0.copy_(torch.as_tensor(np.asarray(xs, np.float32)))
    bt.V.copy_(torch.as_tensor(np.concatenate(Vs).astype(np.float32)))


@pytest.mark.parametrize("rb", [128, 64])
def test_batch_steps_vs_oracle(S, orc, ib, rb):
    bt = S.Batch(ib, block_rollouts=rb)
    B = bt.B
    models = [orc.Model(ib.params[i], ib.tracks[i]) for i in range(B)]
    xs = [ib.x0[i].astype(np.float64) for i in range(B)]
    Vs = [np.zeros((bt.T[i], 2)) for i in range(B)]
    flips = 0
    for n in range(3):
        _set_state(bt, xs, Vs)
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, n, 10)
        st, bits = S.smppi_batch_sync_status(bt.b)
        assert st in (S.OK, S.ERR_STALLED), (st, bits)
        Vg, Vsg, xg = bt.split(bt.V), bt.split(bt.V_safe), bt.x0.cpu().numpy()
        x_next, V_next = [], []
        for i in range(B):
            m = models[i]
            V32 = Vs[i].astype(np.float32)
            x32 = xs[i].astype(np.float32)
            So, Vp = orc.mppi_step(m, x32, V32, n, i, nthreads=8)
            _, om = orc.update(m, So, V32, n, i)
            eps = orc.noise_block(m, n, i, range(m.K))
            tol = update_bound(So, eps, om, Vp, V32, ib.params[i]["lam"])
            Vsh = orc.shift(m, Vp)
            tol_sh = np.concatenate([tol[1:], tol[-1:]])
            assert np.all(np.abs(Vg[i] - Vsh) <= tol_sh), (n, i, np.abs(Vg[i] - Vsh).max())
            Vso, mer, sto, ito = orc.repair(m, x32, Vp.astype(np.float32), 10)
            if np.max(np.abs(Vsg[i] - Vso)) > V_REP:
                flips += 1
            else:
                xo = orc.apply(m, x32, Vso[0], n, i)
                assert rel_err(xg[i], xo) <= X_REL, (n, i)
            x_next.append(orc.apply(m, x32, Vso[0], n, i))
            V_next.append(Vsh)
        xs, Vs = x_next, V_next
    assert flips <= 2
    bt.close()


def test_batch_graph_equals_steps_and_autotune(S, ib):
    bt = S.Batch(ib, block_rollouts=0)      # autotuned at the first step
    x_init = bt.x0.clone()
    for n in range(3):
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, n, 10)
    S.smppi_batch_sync_status(bt.b)
    rb, grid = S.smppi_batch_config(bt.b)
    assert rb in (64, 128, 256) and grid >= 1
    ref = (bt.x0.clone(), bt.V.clone(), bt.V_safe.clone())
    bt.x0.copy_(x_init)
    bt.V.zero_()
    S.smppi_batch_loop(bt.b, bt.x0, bt.V, bt.V_safe, 0, 10, 3)
    S.smppi_batch_sync_status(bt.b)
    assert torch.equal(bt.x0, ref[0]) and torch.equal(bt.V, ref[1])
    assert torch.equal(bt.V_safe, ref[2])
    bt.close()


def test_batch_matches_single_problem_path(S, ib):
    # problem i of the batch == the handle path with instance index i
    bt = S.Batch(ib, block_rollouts=128)
    S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, 0, 10)
    S.smppi_batch_sync_status(bt.b)
    Vg, Vsg, xg = bt.split(bt.V), bt.split(bt.V_safe), bt.x0.cpu().numpy()
    for i in (0, 5, 11):
        ctl = S.Controller(ib.params[i], ib.tracks[i])
        x0 = ctl.tensor(ib.x0[i]); V = ctl.tensor(np.zeros((bt.T[i], 2), np.float32))
        Vs = torch.empty_like(V)
        S.smppi_shield_update(ctl.h, x0, V, Vs, 0, i, 10)
        ctl.sync_status()
        assert np.max(np.abs(V.cpu().numpy() - Vg[i])) <= 1e-5
        assert np.max(np.abs(Vs.cpu().numpy() - Vsg[i])) <= 1e-4
        assert rel_err(xg[i], x0.cpu().numpy()) <= 1e-5
        ctl.close()
    bt.close()


@pytest.mark.parametrize("n_rep,c_cbf", [(0, 0.0), (10, 1000.0)])
def test_batch_monitor_vs_oracle(S, orc, n_rep, c_cbf):
    # safety monitor (executed steps that break the DCBF condition / leave the track)
    # against the oracle's own closed loop, one step at a time: the oracle's state
    # goes to the GPU (oracle -> GPU only), one batch update runs, and the monitor's
    # counts for that step are compared with the condition evaluated on the
    # oracle's executed step; decisions within 1e-3 of the threshold, and steps
    # whose executed control differs (a line-search flip), are skipped
    ib = I.uneven_instances(n_inst=6, seed=11, K_lo=64, K_hi=256, T_lo=20, T_hi=30,
                            w_lo=1.0, w_hi=1.5, C_cbf=c_cbf, **I.HARSH)
    bt = S.Batch(ib, block_rollouts=64)
    B = bt.B
    models = [orc.Model(ib.params[i], ib.tracks[i]) for i in range(B)]
    xs = [ib.x0[i].astype(np.float64) for i in range(B)]
    Vs = [np.zeros((bt.T[i], 2)) for i in range(B)]
    a = 1.0 - float(np.float32(ib.params[0]["alpha"]))
    checked = mism = viol_seen = flips = 0
    for n in range(30):
        _set_state(bt, xs, Vs)
        S.smppi_batch_monitor(bt.b, B, reset=True)
        S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, n, n_rep)
        st, bits = S.smppi_batch_sync_status(bt.b)
        assert st in (S.OK, S.ERR_STALLED), (st, bits)
        viol, out = S.smppi_batch_monitor(bt.b, B, reset=True)
        v0_gpu = [v[0] for v in bt.split(bt.V_safe)]
        for i in range(B):
            m = models[i]
            x32, V32 = xs[i].astype(np.float32), Vs[i].astype(np.float32)
            _, Vp = orc.mppi_step(m, x32, V32, n, i, nthreads=8)
            v_exec = Vp[0]
            if n_rep:
                v_exec = orc.repair(m, x32, Vp.astype(np.float32), n_rep)[0][0]
            x1 = orc.apply(m, x32, v_exec, n, i)
            if np.max(np.abs(v0_gpu[i] - v_exec)) > 1e-4:
                flips += 1          # a line-search decision differs: another executed step
                xs[i], Vs[i] = x1, orc.shift(m, Vp)
                continue
            seg, d2 = orc.track_nearest(m, x32[3], x32[4])
            h0 = orc.h(m, d2)
            _, d21 = orc.track_follow(m, seg, x1[3], x1[4])
            h1 = orc.h(m, d21)
            if abs(h1 - a * h0) > 1e-3 * (abs(h0) + 1.0):
                checked += 1
                mism += int(viol[i]) != int(h1 < a * h0)
                viol_seen += int(h1 < a * h0)
            if abs(h1) > 1e-3:
                checked += 1
                mism += int(out[i]) != int(h1 < 0.0)
            xs[i], Vs[i] = x1, orc.shift(m, Vp)
    print("monitor (n_repair %d): %d decisions checked, %d mismatches, %d violations, %d flips"
          % (n_rep, checked, mism, viol_seen, flips))
    assert checked >= 300 and mism == 0 and flips <= 6
    bt.close()
