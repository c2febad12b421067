"""Pins of the oracle's repair gradient and safety shield (Eq. 22, Alg. 1).

  * the forward-mode (dual number) gradient agrees with central finite
    differences (h = 1e-4, FP64) on the smooth running cost and, away from the
    kinks of max(0, .) and of the clamp (derivative 0 on the inactive side),
    on the CBF objective;
  * an already-safe sequence has zero objective and zero gradient and is a
    fixed point of the shield (the objective of Eq. 22 is 0 iff the CBF
    condition holds on every pair);
  * Armijo backtracking never increases the merit; repair reduces violations;
  * the disturbed closed loop (Eq. 26) and the warm-start shift.
"""
import numpy as np
import pytest

from paper_2302_11719_gb300 import inputs as I


@pytest.fixture(scope="module")
def seqs():
    return I.near_boundary_sequences(n_seq=64, T=40, seed=1)


@pytest.fixture(scope="module")
def model(orc, seqs):
    return orc.Model(seqs.params, seqs.track)


def _fd(orc, m, x0, V, w_run, w_cbf, h=1e-4):
    g = np.zeros((m.T, 2))
    Vd = V.astype(np.float64)
    for t in range(m.T):
        for j in range(2):
            Vp = Vd.copy(); Vp[t, j] += h
            Vm = Vd.copy(); Vm[t, j] -= h
            g[t, j] = (orc.cost(m, x0, Vp, None, w_run, w_cbf) -
                       orc.cost(m, x0, Vm, None, w_run, w_cbf)) / (2 * h)
    return g


def _kink_free(orc, m, x0, V, margin=1e-3):
    """No CBF argument within `margin` of 0 and no control within margin of a bound
    (also for the +-h perturbations of the finite difference)."""
    Vd = V.astype(np.float64)
    lo, hi = np.array([-0.5, -1.0]), np.array([0.5, 1.0])
    if np.any(np.abs(Vd - lo) < margin) or np.any(np.abs(Vd - hi) < margin):
        return False
    _, traj, _ = orc.rollout(m, x0, Vd, noisy=False)
    seg, d2 = orc.track_nearest(m, traj[0][3], traj[0][4])
    hs = [orc.h(m, d2)]
    for x in traj[1:]:
        seg, d2 = orc.track_follow(m, seg, x[3], x[4])
        hs.append(orc.h(m, d2))
    a = 1 - float(np.float32(0.3))
    args = np.array([a * hs[i] - hs[i + 1] for i in range(len(hs) - 1)])
    return bool(np.all(np.abs(args) > margin))


def test_grad_running_cost_matches_fd(orc, model, seqs):
    for i in range(6):
        J, g = orc.cost_grad(model, seqs.x0[i], seqs.V[i], None, 1.0, 0.0)
        gfd = _fd(orc, model, seqs.x0[i], seqs.V[i], 1.0, 0.0)
        lo, hi = np.array([-0.5, -1.0]), np.array([0.5, 1.0])
        inside = (seqs.V[i] > lo + 1e-3) & (seqs.V[i] < hi - 1e-3)
        assert np.linalg.norm((g - gfd)[inside]) <= 1e-6 * max(1.0, np.linalg.norm(gfd[inside]))
        assert J == pytest.approx(orc.cost(model, seqs.x0[i], seqs.V[i], None, 1.0, 0.0), rel=1e-14)


def test_grad_cbf_matches_fd_away_from_kinks(orc, model, seqs):
    checked = 0
    for i in range(seqs.x0.shape[0]):
        if not _kink_free(orc, model, seqs.x0[i], seqs.V[i]):
            continue
        J, g = orc.cost_grad(model, seqs.x0[i], seqs.V[i], None, 1.0, 1.0)
        gfd = _fd(orc, model, seqs.x0[i], seqs.V[i], 1.0, 1.0)
        assert np.linalg.norm(g - gfd) <= 1e-6 * max(1.0, np.linalg.norm(gfd))
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3


def test_grad_zero_outside_repair_horizon(orc, model, seqs):
    J, g = orc.cost_grad(model, seqs.x0[0], seqs.V[0], 10, 0.0, 1.0)
    assert np.all(g[10:] == 0)


def test_safe_sequence_is_fixed_point(orc):
    pr = I.single_problem(K=16, T=30)
    m = orc.Model(pr.params, pr.track)
    # steer along the centreline curvature at theta = 0 from the centre: stays safe
    V = np.zeros((30, 2), np.float32)
    V[:, 0] = np.arctan(0.57 / 7.2)
    P = orc.merit(m, pr.x0, V)
    assert P == 0.0
    J, g = orc.cost_grad(m, pr.x0, V, None, 0.0, 1.0)
    assert J == 0.0 and np.all(g == 0)
    Vs, mer, st, it = orc.repair(m, pr.x0, V, 5)
    assert st == 0 and it == 0 and np.all(mer == 0) and np.array_equal(Vs, V)


def _violations(orc, m, x0, V):
    _, traj, _ = orc.rollout(m, x0, np.asarray(V, np.float64), noisy=False)
    seg, d2 = orc.track_nearest(m, traj[0][3], traj[0][4])
    hs = [orc.h(m, d2)]
    for x in traj[1:]:
        seg, d2 = orc.track_follow(m, seg, x[3], x[4])
        hs.append(orc.h(m, d2))
    a = 1 - float(np.float32(0.3))
    return sum(1 for i in range(len(hs) - 1) if hs[i + 1] < a * hs[i])


def test_armijo_repair_monotone_and_effective(orc, model, seqs):
    improved = 0
    for i in range(12):
        P0 = orc.merit(model, seqs.x0[i], seqs.V[i])
        Vs, mer, st, it = orc.repair(model, seqs.x0[i], seqs.V[i], 20, mode=1)
        assert mer[0] == pytest.approx(P0)
        assert np.all(np.diff(mer) <= 1e-9 * (1 + mer[:-1]))       # never increases
        assert np.all(Vs >= [-0.5, -1.0]) and np.all(Vs <= [0.5, 1.0])
        assert orc.merit(model, seqs.x0[i], Vs) == pytest.approx(mer[-1], rel=1e-12)
        if P0 > 0:
            assert _violations(orc, model, seqs.x0[i], Vs) <= _violations(orc, model, seqs.x0[i],
                                                                        seqs.V[i])
            improved += mer[-1] < 0.5 * P0
    assert improved >= 3


def test_fixed_step_mode(orc, model, seqs):
    i = next(i for i in range(64) if orc.merit(model, seqs.x0[i], seqs.V[i]) > 0)
    Vs, mer, st, it = orc.repair(model, seqs.x0[i], seqs.V[i], 1, mode=0, delta=1e-5)
    _, g = orc.cost_grad(model, seqs.x0[i], seqs.V[i], None, 0.0, 1.0)
    ref = np.clip(seqs.V[i] - 1e-5 * g, [-0.5, -1.0], [0.5, 1.0])
    assert np.allclose(Vs, ref, atol=1e-15)


def test_apply_and_shift(orc):
    pr = I.closed_loop_plain()
    m = orc.Model(pr.params, pr.track)
    x0 = pr.x0.astype(np.float64)
    v0 = np.array([0.1, 0.4])
    nodist = m.with_(dist_sigma=(0.0, 0.0))
    assert np.array_equal(orc.apply(nodist, x0, v0, 3), orc.step(m, x0, v0))
    w = np.array([orc.disturbance(m, n) for n in range(20000)])
    assert np.all(w[:, [0, 3, 4, 5]] == 0)
    assert np.all(np.abs(w[:, 1:3].mean(axis=0)) < 5 * 0.3 / np.sqrt(len(w)))
    assert np.all(np.abs(w[:, 1:3].std(axis=0) - 0.3) < 5 * 0.3 / np.sqrt(2 * len(w)))
    Vp = np.arange(2 * m.T, dtype=np.float64).reshape(m.T, 2)
    Vs = orc.shift(m, Vp)
    assert np.array_equal(Vs[:-1], Vp[1:]) and np.array_equal(Vs[-1], Vp[-1])
