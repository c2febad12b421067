"""Pins of the oracle's MPPI update (Eq. 10-12, Eq. 20, Alg. 2).

  * normalised weights sum to 1 (Eq. 11);
  * the min-shift does not change the solution: V+ is invariant under S -> S + c;
  * lambda -> 0 selects the arg-min sample: V+ = clamp(V + eps_argmin);
  * lambda -> infinity gives the plain sample mean of eps;
  * Sigma -> 0: every rollout is the nominal (noise-free) rollout and V+ = V;
  * the nominal rollout is the iterate of the one-step map f (Eq. 1);
  * rollouts are independent of the thread count and of each other.
"""
import numpy as np
import pytest

from paper_2302_11719_gb300 import inputs as I


@pytest.fixture(scope="module")
def prob():
    return I.single_step_small()


@pytest.fixture(scope="module")
def model(orc, prob):
    return orc.Model(prob.params, prob.track)


@pytest.fixture(scope="module")
def step0(orc, model, prob):
    return orc.mppi_step(model, prob.x0, prob.V, nthreads=2)


def test_weights_sum_to_one(orc, model, prob, step0):
    S, _ = step0
    _, om = orc.update(model, S, prob.V)
    assert om.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.all(om >= 0)
    assert om.argmax() == S.argmin()


def test_shift_invariance(orc, model, prob, step0):
    S, vp = step0
    for c in (-1234.5, 1e3, 7.25):
        vp2, _ = orc.update(model, S + c, prob.V)
        assert np.allclose(vp2, vp, atol=1e-13)


def test_lambda_zero_selects_argmin(orc, model, prob):
    V = np.full((prob.T, 2), 0.05, np.float32)
    m0 = model.with_(lam=1e-6, gamma=0.0)
    S, vp = orc.mppi_step(m0, prob.x0, V)
    k = int(S.argmin())
    eps = orc.noise_block(m0, 0, 0, [k])[0]
    ref = np.clip(V + eps, [-0.5, -1.0], [0.5, 1.0])
    assert np.allclose(vp, ref, atol=1e-12)


def test_lambda_infinity_is_mean(orc, model, prob, step0):
    S, _ = step0
    m_inf = model.with_(lam=1e30)
    vp, om = orc.update(m_inf, S, prob.V)
    assert np.allclose(om, 1.0 / model.K, rtol=1e-9)
    eps = orc.noise_block(model, 0, 0, range(model.K))
    ref = np.clip(prob.V + eps.mean(axis=0), [-0.5, -1.0], [0.5, 1.0])
    assert np.allclose(vp, ref, atol=1e-12)


def test_zero_noise_reproduces_nominal(orc, model, prob):
    V = np.stack([0.1 * np.sin(np.arange(prob.T) / 5), 0.3 * np.ones(prob.T)], 1).astype(np.float32)
    m0 = model.with_(sigma=(1e-19, 1e-19), K=16)
    S, vp = orc.mppi_step(m0, prob.x0, V)
    assert np.allclose(vp, V, atol=1e-15)
    Snom, traj_nom, _ = orc.rollout(m0, prob.x0, V, noisy=False)
    assert np.allclose(S, Snom, rtol=1e-12)
    for k in (0, 5, 15):
        _, traj, _ = orc.rollout(m0, prob.x0, V, k=k)
        assert np.allclose(traj, traj_nom, atol=1e-12)
    # the nominal rollout iterates x_{t+1} = f(x_t, v_t)
    x = prob.x0.astype(np.float64)
    for t in range(prob.T):
        x = orc.step(m0, x, V[t])
        assert np.allclose(x, traj_nom[t + 1], atol=1e-12)


def test_rollout_independent_of_threads_and_order(orc, model, prob, step0):
    S, vp = step0
    S4, vp4 = orc.mppi_step(model, prob.x0, prob.V, nthreads=4)
    assert np.array_equal(S, S4) and np.array_equal(vp, vp4)
    for k in (0, 17, 255):
        Sk, _, _ = orc.rollout(model, prob.x0, prob.V, k=k)
        assert Sk == S[k]


def test_control_cost_term(orc, model, prob):
    # S(gamma) - S(0) = gamma sum_t v_t' Sigma^-1 (v_t + eps_t)
    V = np.full((prob.T, 2), [0.02, 0.1], np.float32)
    s0, _, eps = orc.rollout(model.with_(gamma=0.0), prob.x0, V, k=3)
    s1, _, _ = orc.rollout(model.with_(gamma=2.0), prob.x0, V, k=3)
    sig = np.array([np.float32(0.15), np.float32(0.3)], np.float64)
    ctl = np.sum(V.astype(np.float64) * (V + eps) / sig ** 2)
    assert s1 - s0 == pytest.approx(2.0 * ctl, rel=1e-9)


def test_first_cbf_term_uses_x0_twice(orc, model, prob):
    # Eq. 20 with z_0 = (x_0, x_0): C max(-alpha h(x0), 0) -> C alpha |h| outside the track
    x0 = prob.x0.copy()
    x0[3] += 2.5          # 2.5 m outside the centreline at theta = 0
    m1 = model.with_(T=1, gamma=0.0, q_v=0.0, q_d=0.0, sigma=(1e-19, 1e-19))
    V = np.zeros((1, 2), np.float32)
    S, traj, _ = orc.rollout(m1, x0, V, noisy=False)
    _, d2_0 = orc.track_nearest(m1, x0[3], x0[4])
    seg, d2_1 = orc.track_nearest(m1, traj[1][3], traj[1][4])
    h0, h1 = 4.0 - d2_0, 4.0 - d2_1
    a = float(np.float32(0.3))
    expect = 1000 * max(-a * h0, 0) + 1000 * max((1 - a) * h0 - h1, 0)
    assert S == pytest.approx(expect, rel=1e-9)
    assert expect > 0
