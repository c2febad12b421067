"""Pins of the oracle's curvilinear state variant (the (s, e_y, e_psi) state of
the paper's AutoRally model, Sec. VI-A, on the curvature of the centreline's
turning angles, Frenet kinematics).

  * the curvature table of a regular polygon inscribed in a circle of radius R
    is the closed form (2 pi / n) / chord everywhere, and the track length is
    n chords; traversed clockwise, the samples change sign;
  * on the ellipse track the table follows the ellipse's analytic curvature
    ab / (a^2 sin^2 t + b^2 cos^2 t)^(3/2) at the same arc lengths (positive:
    the counter-clockwise centreline turns left), and so does kappa(s), the
    interpolation the model evaluates, at arbitrary arc lengths (between the
    stations, across the wrap, whole laps forward and backward);
  * on the ellipse, where the curvature varies, the curvilinear and Cartesian
    models agree in (s, e_y, e_psi) with respect to the exact ellipse to first
    order in dt;
  * on a circle the curvilinear model and the Cartesian model, started on the
    centreline along the tangent and driven by the same controls, give the same
    (s, e_y, e_psi) (the Cartesian state converted exactly), with a difference
    that halves with dt (the two explicit Euler schemes agree to first order);
    the velocity states are identical;
  * the rollout cost takes e_y^2 from the state's own e_y;
  * the dual-number gradient of the repair objective through the Frenet
    kinematics and kappa(s) equals central finite differences away from the
    kinks, and the Armijo repair on the curvilinear state never increases the
    merit and makes most near-edge sequences safe;
  * the BFGS repair (mode 2) on the curvilinear state: its first
    iteration is the gradient repair's (H is unset), its merit never
    increases, its iterates stay in the control box, and ten iterations make
    at least half of the unsafe near-edge sequences safe.
"""
import numpy as np
import pytest

from paper_2302_11719_gb300 import inputs as I


def _circle(R, n):
    th = 2 * np.pi * np.arange(n) / n
    return np.stack([R * np.cos(th), R * np.sin(th)], 1).astype(np.float32)


def _curv(params):
    p = dict(params)
    p["state_kind"] = 1
    return p


def test_curvature_regular_polygon(orc):
    R, n = 10.0, 256
    m = orc.Model(_curv(I.make_params(K=1, T=10)), _circle(R, n))
    k, L = orc.curvature_table(m)
    chord = 2 * R * np.sin(np.pi / n)
    assert np.max(np.abs(k / ((2 * np.pi / n) / chord) - 1)) < 5e-4   # float32 vertices
    assert abs(L / (n * chord) - 1) < 1e-7


def test_curvature_sign_follows_orientation(orc):
    # the same polygon traversed clockwise turns right at every vertex: the
    # samples change sign, the length does not
    R, n = 10.0, 256
    ccw = _circle(R, n)
    k1, L1 = orc.curvature_table(orc.Model(_curv(I.make_params(K=1, T=10)), ccw))
    k2, L2 = orc.curvature_table(orc.Model(_curv(I.make_params(K=1, T=10)), ccw[::-1].copy()))
    assert np.all(k1 > 0) and np.all(k2 < 0)
    assert np.allclose(k2, -k1[0], rtol=5e-4) and abs(L2 / L1 - 1) < 1e-12


def test_curvature_ellipse_analytic(orc):
    a, b, n = 20.0, 12.0, 1024
    tr = I.ellipse_track(a, b, n)
    m = orc.Model(_curv(I.make_params(K=1, T=10)), tr)
    k, L = orc.curvature_table(m)
    seg = np.hypot(*(np.roll(tr, -1, 0) - tr).astype(np.float64).T)
    st = np.concatenate([[0.0], np.cumsum(seg)])
    t = np.interp(np.arange(n) * L / n, st, 2 * np.pi * np.arange(n + 1) / n)
    ka = a * b / (a * a * np.sin(t) ** 2 + b * b * np.cos(t) ** 2) ** 1.5
    assert np.all(k > 0)
    assert np.max(np.abs(k / ka - 1)) < 1e-2
    assert np.mean(np.abs(k / ka - 1)) < 2e-3


def _ellipse_curv_model(orc):
    a, b, n = 20.0, 12.0, 1024
    tr = I.ellipse_track(a, b, n)
    m = orc.Model(_curv(I.make_params(K=1, T=10)), tr)
    seg = np.hypot(*(np.roll(tr, -1, 0) - tr).astype(np.float64).T)
    st = np.concatenate([[0.0], np.cumsum(seg)])
    return m, a, b, n, st


def _ellipse_kappa(a, b, n, st, s):
    """Analytic curvature of the ellipse at the parameter whose polyline arc
    length is s (0 <= s < L)."""
    t = np.interp(s, st, 2 * np.pi * np.arange(n + 1) / n)
    return a * b / (a * a * np.sin(t) ** 2 + b * b * np.cos(t) ** 2) ** 1.5


def test_kappa_at_interpolates_ellipse_curvature(orc):
    """kappa(s), the function the curvilinear model evaluates, at arbitrary arc
    lengths (between the stations, in the last interval that wraps to sample 0,
    shifted by whole laps forward and backward) against the ellipse's analytic
    curvature.  The interpolation error is below 0.3 %; taking one station's
    sample instead of interpolating would miss by 0.8 % between stations."""
    m, a, b, n, st = _ellipse_curv_model(orc)
    k, L = orc.curvature_table(m)
    rng = np.random.default_rng(5)
    s = rng.uniform(0.0, L, 3000)
    ka = _ellipse_kappa(a, b, n, st, s)
    kk = np.array([orc.kappa_at(m, x) for x in s])
    assert np.max(np.abs(kk / ka - 1)) < 4e-3
    assert np.mean(np.abs(kk / ka - 1)) < 1e-3
    # midway between stations, where a wrong station index or slope errs most
    mid = (np.arange(n) + 0.5) * L / n
    kmid = np.array([orc.kappa_at(m, x) for x in mid])
    assert np.max(np.abs(kmid / _ellipse_kappa(a, b, n, st, mid) - 1)) < 4e-3
    # the last interval interpolates towards sample 0 (the wrap)
    last = np.linspace((n - 1) * L / n, L, 25, endpoint=False)
    kl = np.array([orc.kappa_at(m, x) for x in last])
    assert np.max(np.abs(kl / _ellipse_kappa(a, b, n, st, last) - 1)) < 4e-3
    # periodic in s with period L, for s >= L and s < 0
    for shift in (L, 3 * L, -L, -2 * L):
        ks = np.array([orc.kappa_at(m, x + shift) for x in s[:300]])
        assert np.max(np.abs(ks - kk[:300])) <= 1e-12 * np.max(np.abs(kk))


def _ellipse_frenet(a, b, X, Y, psi, t):
    """(s, e_y, e_psi) of a Cartesian pose with respect to the exact ellipse
    (a cos t, b sin t): the foot point by Newton from parameter t, the arc
    length from t = 0 by quadrature, e_y positive to the left."""
    from scipy.integrate import quad
    for _ in range(50):
        ex, ey = a * np.cos(t) - X, b * np.sin(t) - Y
        dx, dy = -a * np.sin(t), b * np.cos(t)
        t -= (ex * dx + ey * dy) / (dx * dx + dy * dy - ex * a * np.cos(t) - ey * b * np.sin(t))
    ex, ey = a * np.cos(t), b * np.sin(t)
    dx, dy = -a * np.sin(t), b * np.cos(t)
    nn = np.hypot(dx, dy)
    s = quad(lambda u: np.hypot(a * np.sin(u), b * np.cos(u)), 0.0, t)[0]
    e_psi = (psi - np.arctan2(dy, dx) + np.pi) % (2 * np.pi) - np.pi
    return (s, (-(X - ex) * dy + (Y - ey) * dx) / nn, e_psi), t


def _ellipse_runs(orc, dt, tend=1.0):
    a, b, n = 20.0, 12.0, 1024
    tr = I.ellipse_track(a, b, n)
    T = int(round(tend / dt))
    pc = I.make_params(K=1, T=T, dt=dt, half_width=2.0)
    mc, mk = orc.Model(pc, tr), orc.Model(_curv(pc), tr)
    t = np.arange(T) * dt
    V = np.stack([0.08 + 0.05 * np.sin(3 * t), 0.3 * np.cos(2 * t)], 1)
    _, tc, _ = orc.rollout(mc, np.array([5.0, 0, 0, a, 0, np.pi / 2]), V, noisy=False)
    _, tk, _ = orc.rollout(mk, np.array([5.0, 0, 0, 0, 0, 0]), V, noisy=False)
    conv, tp = [], 0.0
    for row in tc:
        f, tp = _ellipse_frenet(a, b, row[3], row[4], row[5], tp)
        conv.append(f)
    return (np.abs(np.array(conv) - tk[:, 3:6]).max(0), np.abs(tc[:, :3] - tk[:, :3]).max(),
            np.abs(tk[:, 4]).max())


def test_curvilinear_matches_cartesian_on_ellipse(orc):
    """Where the curvature varies (the first 5 m from the end of the major axis,
    kappa from 0.139 /m down): the curvilinear model on the interpolated kappa(s)
    and the Cartesian model on the polyline, same start and controls, agree in
    (s, e_y, e_psi) against the exact ellipse to first order in dt (each
    halving of dt halves the gap; a wrong kappa(s) would leave a gap that does
    not shrink), with identical velocity states."""
    e4, dv4, _ = _ellipse_runs(orc, 4e-3)
    e2, dv2, _ = _ellipse_runs(orc, 2e-3)
    e1, dv1, ey_max = _ellipse_runs(orc, 1e-3)
    assert dv1 == 0.0 and dv2 == 0.0 and dv4 == 0.0
    assert ey_max > 0.3                              # the path really leaves the centreline
    assert e1[0] < 5e-4 and e1[1] < 2e-3 and e1[2] < 2e-4
    for hi, lo in ((e4, e2), (e2, e1)):
        r = hi / lo
        assert np.all((r[:2] > 1.7) & (r[:2] < 2.3)), r
        assert 1.5 < r[2] < 2.6, r


def _circle_runs(orc, dt, R=10.0, n=256, tend=0.5):
    T = int(round(tend / dt))
    pc = I.make_params(K=1, T=T, dt=dt, half_width=2.0)
    mc, mk = orc.Model(pc, _circle(R, n)), orc.Model(_curv(pc), _circle(R, n))
    t = np.arange(T) * dt
    V = np.stack([0.08 + 0.05 * np.sin(3 * t), 0.3 * np.cos(2 * t)], 1)
    _, tc, _ = orc.rollout(mc, np.array([5.0, 0, 0, R, 0, np.pi / 2]), V, noisy=False)
    _, tk, _ = orc.rollout(mk, np.array([5.0, 0, 0, 0, 0, 0]), V, noisy=False)
    th = np.unwrap(np.arctan2(tc[:, 4], tc[:, 3]))
    conv = np.stack([R * th, R - np.hypot(tc[:, 3], tc[:, 4]), tc[:, 5] - (th + np.pi / 2)], 1)
    return np.abs(conv - tk[:, 3:6]).max(0), np.abs(tc[:, :3] - tk[:, :3]).max()


def test_curvilinear_matches_cartesian_on_circle(orc):
    e2, dv2 = _circle_runs(orc, 2e-3)
    e1, dv1 = _circle_runs(orc, 1e-3)
    assert dv1 == 0.0 and dv2 == 0.0                 # (v_x, v_y, r) do not depend on the pose
    assert e1[0] < 2e-4 and e1[1] < 2e-3 and e1[2] < 1e-4
    ratio = e2[:2] / e1[:2]                          # first-order agreement in s and e_y
    assert np.all((ratio > 1.7) & (ratio < 2.3)), ratio
    assert e1[1] > 1e-5                              # the trajectory really leaves the centreline


def test_curvilinear_cost_uses_e_y(orc):
    pr = I.single_problem(K=1, T=40)
    p = _curv(pr.params)
    m = orc.Model(p, pr.track)
    x0 = np.array([6.0, 0.2, 0.1, 3.0, 0.7, 0.05])
    V = np.tile([[0.05, 0.4]], (40, 1))
    S, traj, _ = orc.rollout(m, x0, V, noisy=False)
    w2 = np.float32(p["half_width"]) ** 2
    a1 = 1 - float(np.float32(p["alpha"]))
    ey2 = traj[:, 4] ** 2
    h = w2 - ey2
    q = float(np.float32(p["q_v"])) * (traj[:, 0] - float(np.float32(p["v_target"]))) ** 2 + \
        float(np.float32(p["q_d"])) * ey2 / w2
    cbf = np.maximum(a1 * np.concatenate([[h[0]], h[:-1]]) - h, 0) * float(np.float32(p["C_cbf"]))
    gam = float(np.float32(p["gamma"]))
    sig = np.array(p["sigma"], np.float32).astype(np.float64)
    ctrl = gam * np.sum(V * V / sig ** 2)
    assert S == pytest.approx(q.sum() + cbf.sum() + ctrl, rel=1e-12)
    assert np.max(np.abs(traj[:, 4])) > 0.5          # e_y enters, not a polyline distance


def _curv_sequences(n=8, T=40, seed=3):
    """Curvilinear starts near the track edge heading toward it, and smooth
    control sequences that steer further out (the repair's inputs)."""
    sb = I.near_edge_curvilinear(n, T, seed)
    return sb.params, sb.track, sb.x0.astype(np.float64), sb.V.astype(np.float64)


def _fd(orc, m, x0, V, w_run, w_cbf, h=1e-4):
    g = np.zeros_like(V)
    for t in range(V.shape[0]):
        for j in range(2):
            Vp, Vm = V.copy(), V.copy()
            Vp[t, j] += h
            Vm[t, j] -= h
            g[t, j] = (orc.cost(m, x0, Vp, None, w_run, w_cbf) -
                       orc.cost(m, x0, Vm, None, w_run, w_cbf)) / (2 * h)
    return g


def test_curvilinear_gradient_matches_fd(orc):
    # the dual-number gradient through the Frenet kinematics and kappa(s), away from
    # the kinks of max(0, .) (derivative 0 on the inactive side)
    p, tr, x0s, Vs = _curv_sequences()
    m = orc.Model(p, tr)
    a1 = 1 - float(np.float32(p["alpha"]))
    w2 = float(np.float32(p["half_width"])) ** 2
    checked = 0
    for i in range(len(x0s)):
        _, traj, _ = orc.rollout(m, x0s[i], Vs[i], noisy=False)
        h = w2 - traj[:, 4] ** 2
        if np.any(np.abs(a1 * h[:-1] - h[1:]) < 1e-3):
            continue
        for w_run, w_cbf in ((1.0, 0.0), (0.0, 1.0), (1.0, 1.0)):
            _, g = orc.cost_grad(m, x0s[i], Vs[i], None, w_run, w_cbf)
            gfd = _fd(orc, m, x0s[i], Vs[i], w_run, w_cbf)
            assert np.linalg.norm(g - gfd) <= 1e-6 * max(1.0, np.linalg.norm(gfd)), (i, w_run, w_cbf)
        checked += 1
    assert checked >= 3


def test_curvilinear_repair_monotone_and_effective(orc):
    p, tr, x0s, Vs = _curv_sequences()
    m = orc.Model(p, tr)
    unsafe, safe_after = 0, 0
    for i in range(len(x0s)):
        Vr, mer, st, it = orc.repair(m, x0s[i], Vs[i], 10)
        assert np.all(np.diff(mer) <= 0.0)
        if mer[0] > 0:
            unsafe += 1
            safe_after += mer[-1] == 0.0
    assert unsafe >= 4 and safe_after >= unsafe // 2


def test_curvilinear_bfgs_first_step_and_descent(orc):
    p, tr, x0s, Vs = _curv_sequences()
    m = orc.Model(p, tr)
    unsafe, safe_after = 0, 0
    for i in range(len(x0s)):
        Va = orc.repair(m, x0s[i], Vs[i], 1, mode=1)[0]
        Vb = orc.repair(m, x0s[i], Vs[i], 1, mode=2)[0]
        assert np.array_equal(Va, Vb)
        Vr, mer, st, it = orc.repair(m, x0s[i], Vs[i], 10, mode=2)
        assert np.all(np.diff(mer) <= 0.0)
        assert np.all((Vr[:, 0] >= -0.5) & (Vr[:, 0] <= 0.5) & (Vr[:, 1] >= -1) & (Vr[:, 1] <= 1))
        if mer[0] > 0:
            unsafe += 1
            safe_after += mer[-1] == 0.0
    assert unsafe >= 4 and safe_after >= unsafe // 2
