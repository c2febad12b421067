"""GPU adjoint, safety shield and closed loop against the FP64 oracle.

  * smppi_cost_grad (checkpointed reverse-mode adjoint) vs the oracle's
    forward-mode dual gradient on near-boundary sequences (T = 100,
    checkpoint every 10): cost within 1e-4 relative, gradient within 1e-3
    relative l2 on sequences with no max(0, .) or clamp kink within 1e-3
    (where the derivative is taken as 0), reported for the rest; checkpointed == full tape exactly;
  * the autograd wrapper returns the same gradient;
  * smppi_repair (Armijo) on the K = 256, T = 50 problem's V+ and on
    near-boundary sequences: repaired controls within 1e-4 of the oracle
    unless a line-search accept/reject decision differs between float32 and
    float64 (counted as a flip, none allowed on the small problem);
  * the closed-loop step (disturbance, warm-start shift) and the whole
    Shield-MPPI update through device buffers, host buffers and a CUDA graph.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import (G_REL, S_REL, V_REP, X_REL, rel_err, repair_compare,  # noqa: E402
                                update_bound)


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


@pytest.fixture(scope="module")
def seqs():
    return I.near_boundary_sequences(n_seq=512, T=100, seed=2)


def kinks(orc, m, x0, V, margin=1e-3):
    Vd = np.asarray(V, np.float64)
    if np.any(np.abs(Vd - [-0.5, -1.0]) < margin) or np.any(np.abs(Vd - [0.5, 1.0]) < margin):
        return True
    _, traj, _ = orc.rollout(m, x0, Vd, noisy=False)
    seg, d2 = orc.track_nearest(m, traj[0][3], traj[0][4])
    hs = [orc.h(m, d2)]
    for x in traj[1:]:
        seg, d2 = orc.track_follow(m, seg, x[3], x[4])
        hs.append(orc.h(m, d2))
    a = 1 - float(np.float32(0.3))
    args = np.array([a * hs[i] - hs[i + 1] for i in range(len(hs) - 1)])
    return bool(np.any(np.abs(args) < margin))


def gpu_cost_grad(S, ctl, x0, V, N, w_run, w_cbf, ck):
    n = x0.shape[0]
    J = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, ctl.T, 2), device="cuda")
    S.smppi_cost_grad(ctl.h, n, ctl.tensor(x0), ctl.tensor(V), N, w_run, w_cbf, ck, J, g)
    assert ctl.sync_status()[0] == S.OK
    return J.cpu().numpy(), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("w_run,w_cbf", [(1.0, 1.0), (0.0, 1.0), (1.0, 0.0)])
def test_cost_grad_vs_oracle(S, orc, seqs, w_run, w_cbf):
    n = 64
    ctl = S.Controller(seqs.params, seqs.track, max_seq=n, checkpoint=10)
    J, g = gpu_cost_grad(S, ctl, seqs.x0[:n], seqs.V[:n], 100, w_run, w_cbf, 10)
    m = orc.Model(seqs.params, seqs.track)
    worst_clean, worst_kink, clean = 0.0, 0.0, 0
    for i in range(n):
        Jo, go = orc.cost_grad(m, seqs.x0[i], seqs.V[i], 100, w_run, w_cbf)
        assert abs(J[i] - Jo) <= S_REL * (abs(Jo) + 1), (i, J[i], Jo)
        e = np.linalg.norm(g[i] - go) / max(np.linalg.norm(go), 1e-12)
        if np.linalg.norm(go) == 0:
            assert np.all(g[i] == 0)
            continue
        if kinks(orc, m, seqs.x0[i], seqs.V[i]):
            worst_kink = max(worst_kink, e)
        else:
            clean += 1
            worst_clean = max(worst_clean, e)
    print("grad rel l2: kink-free max %.2e over %d, near-kink max %.2e" % (worst_clean, clean,
                                                                        worst_kink))
    assert clean >= 8
    assert worst_clean <= G_REL
    ctl.close()


def test_checkpoint_equals_full_tape(S, seqs):
    n = 256
    ctl = S.Controller(seqs.params, seqs.track, max_seq=n, checkpoint=10)
    outs = [gpu_cost_grad(S, ctl, seqs.x0[:n], seqs.V[:n], 100, 1.0, 1.0, ck)
            for ck in (10, -1, 1, 7, 100)]
    for J, g in outs[1:]:
        assert np.array_equal(J, outs[0][0]) and np.array_equal(g, outs[0][1])
    # a shorter sum leaves the tail of the gradient at zero
    J, g = gpu_cost_grad(S, ctl, seqs.x0[:n], seqs.V[:n], 37, 0.0, 1.0, 10)
    assert np.all(g[:, 37:] == 0)
    ctl.close()


def test_autograd_function(S, seqs):
    n = 16
    ctl = S.Controller(seqs.params, seqs.track, max_seq=n, checkpoint=10)
    V = ctl.tensor(seqs.V[:n]).requires_grad_(True)
    x0 = ctl.tensor(seqs.x0[:n])
    J = S.ShieldCost.apply(V, x0, ctl, 1.0, 1.0)
    w = torch.arange(1, n + 1, device="cuda", dtype=torch.float32)
    (J * w).sum().backward()
    Jr, gr = gpu_cost_grad(S, ctl, seqs.x0[:n], seqs.V[:n], 100, 1.0, 1.0, 0)
    assert np.allclose(V.grad.cpu().numpy(), gr * w.cpu().numpy()[:, None, None], rtol=1e-6)
    ctl.close()


def test_repair_small_problem(S, orc):
    pr = I.single_step_small()
    m = orc.Model(pr.params, pr.track)
    # the repair starts from the oracle's V+ of the K = 256, T = 50 step
    _, Vp = orc.mppi_step(m, pr.x0, pr.V, nthreads=8)
    starts = [Vp.astype(np.float32)]
    # and from sequences that leave the track, so that the shield has work to do
    for b in (0.0, -0.05, -0.1, 0.05):
        starts.append(np.tile(np.array([[b, 0.5]], np.float32), (pr.T, 1)))
    x0s = np.tile(pr.x0, (len(starts), 1))
    flips, worst = repair_compare(S, orc, pr.params, pr.track, x0s, np.stack(starts), 10)
    print("K=256 T=50 repair (5 starts, 10 Armijo iterations): %d flips, max |V_safe err| %.2e"
          % (flips, worst))
    assert flips == 0 and worst <= V_REP, (flips, worst)


def test_repair_near_boundary_batch(S, orc, seqs):
    n = 64
    flips, worst = repair_compare(S, orc, seqs.params, seqs.track, seqs.x0[:n], seqs.V[:n], 20)
    print("near-boundary repair: %d flips of %d, worst |dV| %.2e" % (flips, n, worst))
    assert worst <= V_REP
    assert flips <= n // 8


@pytest.mark.parametrize("T,N_r", [(40, 0), (1, 1)])
def test_repair_degenerate_horizons(S, orc, T, N_r):
    # N_r = 0: the objective of Eq. 22 is an empty sum, so P = 0 and nothing
    # changes; T = N_r = 1: a one-step repair
    pr = I.single_problem(K=64, T=T, N_r=N_r)
    rng = np.random.default_rng(T)
    x0 = np.tile(I.centreline_start(20.0, 12.0, 7.0), (4, 1))
    x0[:, 4] += np.array([1.9, -1.9, 1.0, 0.0], np.float32)
    V = np.stack([np.tile([[0.45, 1.0]], (T, 1)), np.tile([[-0.45, 1.0]], (T, 1)),
                  rng.uniform(-0.5, 0.5, (T, 2)), np.zeros((T, 2))]).astype(np.float32)
    flips, worst = repair_compare(S, orc, pr.params, pr.track, x0, V, 5)
    assert flips == 0 and worst <= V_REP, (flips, worst)
    if N_r == 0:
        m = orc.Model(pr.params, pr.track)
        for i in range(4):
            Vo, mo, so, io = orc.repair(m, x0[i], V[i], 5)
            assert io == 0 and np.all(mo == 0.0) and np.array_equal(Vo, V[i].astype(np.float64))


def test_fixed_step_repair(S, orc, seqs):
    n = 8
    ctl = S.Controller(seqs.params, seqs.track, max_seq=n)
    Vout = torch.empty((n, ctl.T, 2), device="cuda")
    S.smppi_repair(ctl.h, n, ctl.tensor(seqs.x0[:n]), ctl.tensor(seqs.V[:n]), Vout, 1, 0, 1e-6)
    assert ctl.sync_status()[0] == S.OK
    m = orc.Model(seqs.params, seqs.track)
    for i in range(n):
        Vo, _, _, _ = orc.repair(m, seqs.x0[i], seqs.V[i], 1, mode=0, delta=1e-6)
        assert np.max(np.abs(Vout[i].cpu().numpy() - Vo)) <= V_REP
    ctl.close()


def test_apply_closed_loop_step(S, orc):
    pr = I.closed_loop_plain()
    ctl = S.Controller(pr.params, pr.track)
    m = orc.Model(pr.params, pr.track)
    rng = np.random.default_rng(1)
    Vp = rng.uniform(-0.4, 0.4, (pr.T, 2)).astype(np.float32)
    for n in (0, 1, 199, 12345):
        x0 = ctl.tensor(pr.x0)
        V = ctl.tensor(Vp)
        S.smppi_apply(ctl.h, x0, V, V, n, 0)     # plain MPPI: execute v0 of V+ itself
        assert ctl.sync_status()[0] == S.OK
        xo = orc.apply(m, pr.x0, Vp[0], n)
        assert rel_err(x0.cpu().numpy(), xo) <= X_REL
        assert np.array_equal(V.cpu().numpy(), orc.shift(m, Vp).astype(np.float32))
    ctl.close()


def test_shield_update_device_host_graph_agree(S):
    pr = I.single_problem(K=4096, T=50)
    ctl = S.Controller(pr.params, pr.track)
    n_up = 5
    # device buffers, one call per update
    x0 = ctl.tensor(pr.x0); V = ctl.tensor(pr.V); Vs = torch.empty_like(V)
    for it in range(n_up):
        S.smppi_shield_update(ctl.h, x0, V, Vs, it, 0, 10)
    assert ctl.sync_status()[0] in (S.OK, S.ERR_STALLED)
    ref = (x0.cpu().numpy(), V.cpu().numpy(), Vs.cpu().numpy())
    # host buffers
    hx = pr.x0.copy(); hV = pr.V.copy(); hVs = np.zeros_like(hV)
    for it in range(n_up):
        S.smppi_shield_update(ctl.h, hx, hV, hVs, it, 0, 10, None, True)
    assert np.array_equal(hx, ref[0]) and np.array_equal(hV, ref[1]) and np.array_equal(hVs, ref[2])
    # CUDA graph replays
    x0 = ctl.tensor(pr.x0); V = ctl.tensor(pr.V); Vs = torch.empty_like(V)
    S.smppi_shield_loop(ctl.h, x0, V, Vs, 0, 0, 10, n_up)
    ctl.sync_status()
    assert np.array_equal(x0.cpu().numpy(), ref[0])
    assert np.array_equal(V.cpu().numpy(), ref[1]) and np.array_equal(Vs.cpu().numpy(), ref[2])
    ctl.close()


@pytest.mark.parametrize("offset,heading", [(1.7, 0.25), (-1.6, -0.3), (0.0, 0.0)])
def test_shield_update_vs_oracle(S, orc, offset, heading):
    # one whole Shield-MPPI update (rollouts, softmin, repair of V+ in the update's
    # last block, closed-loop step) from a state near the boundary and heading out
    # of the track, against the oracle's mppi_step -> repair -> apply -> shift
    pr = I.single_problem(K=512, T=50)
    x0 = pr.x0.copy()
    x0[3] += offset                       # the start (a, 0) has outward normal +X
    x0[5] -= heading                      # heading pi/2 - heading: toward +X for heading > 0
    x0[0] = 6.0
    V = np.tile(np.array([[0.0, 0.3]], np.float32), (pr.T, 1))
    it, inst = 3, 2
    ctl = S.Controller(pr.params, pr.track)
    xg, Vg, Vsg = ctl.tensor(x0), ctl.tensor(V), torch.empty((pr.T, 2), device="cuda")
    S.smppi_shield_update(ctl.h, xg, Vg, Vsg, it, inst, 10)
    st, bits = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), (st, bits)
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, x0, V, it, inst, nthreads=8)
    Vsafe, mer, ost, its = orc.repair(m, x0, Vp.astype(np.float32), 10)
    x1 = orc.apply(m, x0, Vsafe[0], it, inst)
    print("offset %.1f: oracle repair iterations %d, merit %.4g -> %.4g"
          % (offset, its, mer[0], mer[its]))
    _, om = orc.update(m, So, V, it, inst)
    eps = orc.noise_block(m, it, inst, range(m.K))
    tol = update_bound(So, eps, om, Vp, V, pr.params["lam"])
    tol_sh = np.concatenate([tol[1:], tol[-1:]])
    assert np.all(np.abs(Vg.cpu().numpy() - orc.shift(m, Vp)) <= tol_sh)
    assert np.max(np.abs(Vsg.cpu().numpy() - Vsafe)) <= V_REP
    assert rel_err(xg.cpu().numpy(), x1) <= X_REL
    ctl.close()
