"""Closed loop of plain MPPI (no shield, no CBF cost; K = 1024, T = 60) with the
seeded disturbance of Eq. 26, against the FP64 oracle step by step.

The oracle runs its own closed loop for 200 steps.  At every step n its state
(x_n, V_n) is given to the GPU (oracle -> GPU only), one GPU update runs
through smppi_shield_update with no repair, and the GPU's next state and warm
start are compared with the oracle's: x_{n+1} within 1e-4 relative, the
shifted V+ within the update tolerance bound.  The free-running GPU loop is
then run for 2000 steps (CUDA graph) and its CBF violation counts are
reported, next to Shield-MPPI (DCBF cost + 10 repair iterations) on the same
disturbance sequence.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import X_REL, rel_err, update_bound  # noqa: E402


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def test_closed_loop_stepwise_vs_oracle(S, orc):
    pr = I.closed_loop_plain()
    m = orc.Model(pr.params, pr.track)
    n_steps = 200
    xs, Vs = [pr.x0.astype(np.float64)], [np.zeros((pr.T, 2))]
    for n in range(n_steps):
        x32, V32 = xs[-1].astype(np.float32), Vs[-1].astype(np.float32)
        So, Vp = orc.mppi_step(m, x32, V32, n, 0, nthreads=16)
        xs.append(orc.apply(m, x32, Vp[0], n))
        Vs.append(orc.shift(m, Vp))
    ctl = S.Controller(pr.params, pr.track)
    worst_x, worst_v = 0.0, 0.0
    check = list(range(0, n_steps, 10)) + [n_steps - 1]
    for n in range(n_steps):
        x0 = ctl.tensor(xs[n]); V = ctl.tensor(Vs[n]); Vsafe = torch.empty_like(V)
        S.smppi_shield_update(ctl.h, x0, V, Vsafe, n, 0, 0)
        if n not in check:
            continue
        assert ctl.sync_status()[0] == S.OK
        x32, V32 = xs[n].astype(np.float32), Vs[n].astype(np.float32)
        So, Vp = orc.mppi_step(m, x32, V32, n, 0, nthreads=16)
        _, om = orc.update(m, So, V32, n, 0)
        eps = orc.noise_block(m, n, 0, range(m.K))
        tol = update_bound(So, eps, om, Vp, V32, pr.params["lam"])
        tol_sh = np.concatenate([tol[1:], tol[-1:]])
        dv = np.abs(V.cpu().numpy() - Vs[n + 1])
        assert np.all(dv <= tol_sh), (n, dv.max())
        ex = rel_err(x0.cpu().numpy(), xs[n + 1])
        assert ex <= X_REL, (n, ex)
        worst_x, worst_v = max(worst_x, ex), max(worst_v, dv.max())
    print("closed loop, 200 oracle-synced steps: max rel x err %.2e, max |V err| %.2e"
          % (worst_x, worst_v))
    ctl.close()


def _violations(orc, m, traj):
    seg, d2 = orc.track_nearest(m, traj[0][3], traj[0][4])
    hs = [orc.h(m, d2)]
    for x in traj[1:]:
        seg, d2 = orc.track_nearest(m, x[3], x[4])
        hs.append(orc.h(m, d2))
    a = 1 - float(np.float32(0.3))
    pairs = sum(1 for i in range(len(hs) - 1) if hs[i + 1] < a * hs[i] - 1e-9)
    outside = sum(1 for h in hs if h < 0)
    return pairs, outside


def test_closed_loop_2000_steps_violations(S, orc):
    out = {}
    for name, over, n_rep in (("plain MPPI", dict(C_cbf=0.0), 0),
                              ("Shield-MPPI", dict(), 10)):
        pr = I.single_problem(K=1024, T=60, **over)
        m = orc.Model(pr.params, pr.track)
        ctl = S.Controller(pr.params, pr.track)
        x0 = ctl.tensor(pr.x0); V = ctl.tensor(pr.V); Vsafe = torch.empty_like(V)
        traj = [pr.x0.astype(np.float64)]
        for n in range(2000):
            S.smppi_shield_update(ctl.h, x0, V, Vsafe, n, 0, n_rep)
            traj.append(x0.cpu().numpy().astype(np.float64))
        st, bits = ctl.sync_status()
        assert st in (S.OK, S.ERR_STALLED)
        traj = np.array(traj)
        assert np.all(np.isfinite(traj))
        out[name] = _violations(orc, m, traj) + (float(np.mean(traj[:, 0])),)
        ctl.close()
    for k, (pairs, outside, vmean) in out.items():
        print("%s, 2000 steps: CBF-condition violations %d, steps outside the track %d, "
              "mean v_x %.2f m/s" % (k, pairs, outside, vmean))
