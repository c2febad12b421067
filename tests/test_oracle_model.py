"""Pins of the oracle's vehicle model, track distance, cost and DCBF penalty.

Dynamics (single-track model of Sec. VI-A, the equations this implementation fixes):
  * straight running (delta = 0, v_y = r = 0) is a linear ODE that explicit
    Euler integrates exactly: v_x' = v_x + dt 60 a / m, X, Y advance along psi;
  * mirror symmetry about the heading axis (delta, v_y, r, Y, psi -> -);
  * rigid rotation of the pose rotates (X', Y') and leaves the rest unchanged;
  * in the small-slip limit the tyre law Fz sin(C atan(B alpha)) reduces to the
    textbook linear bicycle model with cornering stiffness Fz B C.
Track: distances to a circle and to an ellipse (Newton on the exact curve)
within the polyline's sagitta; tracked projection equals the global nearest
segment inside the track.  DCBF penalty: the hand-worked cases of
tests/golden/cbf_hand_cases.txt (Eq. 17, Eq. 23).
"""
import math
import os

import numpy as np
import pytest

from paper_2302_11719_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def model(orc):
    pr = I.single_step_small()
    return orc.Model(pr.params, pr.track)


def f32(x):
    return float(np.float32(x))


def test_straight_line_euler_exact(orc, model):
    m, dt = f32(21.7), f32(0.02)
    for psi in (0.0, 0.7, -2.0):
        for a in (0.0, 0.5, -1.0):
            x = np.array([5.0, 0.0, 0.0, 3.0, -4.0, psi])
            xn = orc.step(model, x, [0.0, a])
            assert xn[0] == pytest.approx(5.0 + dt * f32(60.0) * a / m, abs=1e-14)
            assert xn[1] == 0.0 and xn[2] == 0.0 and xn[5] == psi
            assert xn[3] == pytest.approx(3.0 + dt * 5.0 * math.cos(psi), abs=1e-14)
            assert xn[4] == pytest.approx(-4.0 + dt * 5.0 * math.sin(psi), abs=1e-14)


def test_mirror_symmetry(orc, model):
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = np.array([rng.uniform(1, 9), rng.normal(0, 0.5), rng.normal(0, 1),
                      rng.normal(0, 10), rng.normal(0, 10), rng.uniform(-3, 3)])
        u = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-1, 1)])
        xm = x * np.array([1, -1, -1, 1, -1, -1])
        um = u * np.array([-1, 1])
        d = orc.deriv(model, x, u)
        dm = orc.deriv(model, xm, um)
        assert np.allclose(dm, d * np.array([1, -1, -1, 1, -1, -1]), rtol=1e-12, atol=1e-12)


def test_pose_rotation_equivariance(orc, model):
    rng = np.random.default_rng(2)
    for _ in range(20):
        x = np.array([rng.uniform(1, 9), rng.normal(0, 0.5), rng.normal(0, 1),
                      rng.normal(0, 10), rng.normal(0, 10), rng.uniform(-3, 3)])
        u = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-1, 1)])
        th = rng.uniform(-3, 3)
        c, s = math.cos(th), math.sin(th)
        xr = x.copy()
        xr[3], xr[4] = c * x[3] - s * x[4], s * x[3] + c * x[4]
        xr[5] = x[5] + th
        d, dr = orc.deriv(model, x, u), orc.deriv(model, xr, u)
        assert np.allclose(dr[[0, 1, 2, 5]], d[[0, 1, 2, 5]], rtol=1e-12, atol=1e-12)
        assert np.allclose(dr[3:5], [c * d[3] - s * d[4], s * d[3] + c * d[4]], atol=1e-12)


def test_linear_tyre_limit(orc, model):
    # Linear bicycle model (e.g. Rajamani, Vehicle Dynamics and Control, ch. 2):
    # alpha_f = delta - (v_y + lf r)/v_x, alpha_r = -(v_y - lr r)/v_x,
    # Fy = C_alpha alpha with C_alpha = Fz B C.
    m_, Iz, lf, lr, g = f32(21.7), f32(1.12), f32(0.34), f32(0.23), f32(9.81)
    B, Ct = 4.0, 1.5
    Fzf, Fzr = m_ * g * lr / (lf + lr), m_ * g * lf / (lf + lr)
    Cf, Cr = Fzf * B * Ct, Fzr * B * Ct
    for scale in (1e-3, 1e-4):
        vx, vy, r, delta = 5.0, 0.3 * scale, -0.7 * scale, 0.5 * scale
        x = np.array([vx, vy, r, 0.0, 0.0, 0.0])
        d = orc.deriv(model, x, [delta, 0.0])
        af, ar = delta - (vy + lf * r) / vx, -(vy - lr * r) / vx
        Fyf, Fyr = Cf * af, Cr * ar
        vy_dot = (Fyr + Fyf) / m_ - vx * r
        r_dot = (lf * Fyf - lr * Fyr) / Iz
        # relative deviation shrinks like the slip squared
        assert abs(d[1] - vy_dot) <= 5 * scale ** 2 * abs(vy_dot) + 1e-15
        assert abs(d[2] - r_dot) <= 5 * scale ** 2 * abs(r_dot) + 1e-15


def test_circle_track_distance(orc):
    R, n = 15.0, 1024
    p = I.make_params()
    trk = I.ellipse_track(R, R, n)
    mdl = orc.Model(p, trk)
    sag = R * (1 - math.cos(math.pi / n)) + 1e-5   # polyline sagitta + float32 rounding
    rng = np.random.default_rng(3)
    for _ in range(200):
        th, rho = rng.uniform(0, 2 * np.pi), rng.uniform(R - 4, R + 4)
        X, Y = rho * math.cos(th), rho * math.sin(th)
        seg, d2 = orc.track_nearest(mdl, X, Y)
        assert abs(math.sqrt(d2) - abs(R - rho)) <= sag


def _ellipse_dist(a, b, X, Y):
    # distance to the exact ellipse: minimise |E(theta) - P|^2 by Newton from a dense grid
    th = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
    d2 = (a * np.cos(th) - X) ** 2 + (b * np.sin(th) - Y) ** 2
    t = th[np.argmin(d2)]
    for _ in range(50):
        ex, ey = a * math.cos(t) - X, b * math.sin(t) - Y
        dx, dy = -a * math.sin(t), b * math.cos(t)
        ddx, ddy = -a * math.cos(t), -b * math.sin(t)
        g = ex * dx + ey * dy
        H = dx * dx + dy * dy + ex * ddx + ey * ddy
        t -= g / H
    return math.hypot(a * math.cos(t) - X, b * math.sin(t) - Y)


def test_ellipse_distance_and_tracking(orc, model):
    a, b, n = 20.0, 12.0, 1024
    # sagitta of a chord of length <= 2 pi a / n on a curve of radius >= b^2 / a
    sag = (2 * math.pi * a / n) ** 2 / (8 * b * b / a) + 1e-5
    rng = np.random.default_rng(4)
    for _ in range(100):
        th = rng.uniform(0, 2 * np.pi)
        tx, ty = -a * math.sin(th), b * math.cos(th)
        nn = math.hypot(tx, ty)
        d = rng.uniform(-2, 2)
        X, Y = a * math.cos(th) - d * ty / nn, b * math.sin(th) + d * tx / nn
        seg, d2 = orc.track_nearest(model, X, Y)
        assert abs(math.sqrt(d2) - _ellipse_dist(a, b, X, Y)) < sag
        # tracked projection from a nearby start reaches the same distance
        for start in (seg - 3, seg + 2, seg):
            s2, dd2 = orc.track_follow(model, start % n, X, Y)
            assert dd2 == pytest.approx(d2, abs=1e-12)


def test_tracked_projection_outside_track(orc, model):
    """The tracked nearest segment (reading c15) followed along continuous paths
    that leave the track by up to twice the half-width, inward and outward: at
    every point it equals the global nearest segment (same squared distance;
    the segment itself up to equal-distance ties).  The ellipse's smallest
    radius of curvature b^2/a = 7.2 m exceeds 2w = 4 m, so no path crosses the
    inner cut locus (the part of the major axis between the centres of
    curvature).  Past it the two differ: a path from the top of the track
    straight down to (0, -1) keeps the top as its (local) nearest point at
    13 m while the bottom, at 11 m, is the global one."""
    a, b, n = 20.0, 12.0, 1024
    rng = np.random.default_rng(11)
    for _ in range(60):
        th = rng.uniform(0, 2 * np.pi)
        tx, ty = -a * math.sin(th), b * math.cos(th)
        nn = math.hypot(tx, ty)
        d_end = rng.choice([-1.0, 1.0]) * rng.uniform(2.0, 4.0)
        seg, _ = orc.track_nearest(model, a * math.cos(th), b * math.sin(th))
        for d in np.linspace(0.0, d_end, 41)[1:]:
            X, Y = a * math.cos(th) - d * ty / nn, b * math.sin(th) + d * tx / nn
            seg, d2 = orc.track_follow(model, seg, X, Y)
            gseg, gd2 = orc.track_nearest(model, X, Y)
            assert d2 == gd2, (th, d)
            assert seg == gseg or orc.seg_dist2(model, gseg, X, Y) == d2
    # past the inner cut locus the tracked and the global projection differ
    seg, _ = orc.track_nearest(model, 0.0, b)
    for Y in np.linspace(b, -1.0, 131)[1:]:
        seg, d2 = orc.track_follow(model, seg, 0.0, Y)
    _, gd2 = orc.track_nearest(model, 0.0, -1.0)
    assert math.sqrt(d2) == pytest.approx(13.0, abs=1e-3)
    assert math.sqrt(gd2) == pytest.approx(11.0, abs=1e-3)


def test_segment_distance_endpoints(orc, model):
    A = model.track[0].astype(np.float64)
    Bp = model.track[1].astype(np.float64)
    D = Bp - A
    # beyond the end point the distance is to the end point
    P = Bp + 0.5 * D / np.linalg.norm(D)
    assert orc.seg_dist2(model, 0, *P) == pytest.approx(0.25, rel=1e-9)
    P = A - 0.3 * D / np.linalg.norm(D)
    assert orc.seg_dist2(model, 0, *P) == pytest.approx(0.09, rel=1e-9)
    # perpendicular offset from the middle
    nrm = np.array([-D[1], D[0]]) / np.linalg.norm(D)
    P = A + 0.5 * D + 1.25 * nrm
    assert orc.seg_dist2(model, 0, *P) == pytest.approx(1.5625, rel=1e-9)


def test_cbf_hand_cases(orc, model):
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "cbf_hand_cases.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for d_prev, d_now, h_prev, h_now, thr, pen in rows:
        assert orc.h(model, d_prev ** 2) == pytest.approx(h_prev, abs=1e-12)
        assert orc.h(model, d_now ** 2) == pytest.approx(h_now, abs=1e-12)
        assert orc.cbf_penalty(model, h_prev, h_now) == pytest.approx(pen, abs=2e-4)


def test_running_cost_values(orc, model):
    assert orc.q(model, [8, 0, 0, 0, 0, 0], 0.0) == 0.0
    # 2 (6 - 8)^2 + 100 * 1 / 4 = 33
    assert orc.q(model, [6, 0, 0, 0, 0, 0], 1.0) == pytest.approx(33.0, abs=1e-5)
    # collision indicator (Eq. 25) only outside the track
    m2 = model.with_(C_obs=50.0)
    assert orc.q(m2, [8, 0, 0, 0, 0, 0], 3.9) == pytest.approx(100 * 3.9 / 4, rel=1e-6)
    assert orc.q(m2, [8, 0, 0, 0, 0, 0], 4.1) == pytest.approx(100 * 4.1 / 4 + 50, rel=1e-6)


def test_property1_forward_invariance(orc, model):
    # Property 1 (Sec. III): if every pair satisfies h_{k+1} >= (1-alpha) h_k then
    # h_k >= (1-alpha)^k h_0 >= 0.  Check on sampled trajectories with zero penalty.
    pr = I.single_step_small()
    hits = 0
    for k in range(64):
        S, traj, _ = orc.rollout(model, pr.x0, pr.V, k=k)
        hs = []
        seg = None
        for x in traj:
            if seg is None:
                seg, d2 = orc.track_nearest(model, x[3], x[4])
            else:
                seg, d2 = orc.track_follow(model, seg, x[3], x[4])
            hs.append(orc.h(model, d2))
        ok = all(hs[i + 1] >= 0.7 * hs[i] for i in range(len(hs) - 1))
        if ok:
            hits += 1
            assert all(hs[i] >= 0.7 ** i * hs[0] - 1e-9 for i in range(len(hs)))
            assert min(hs) >= 0
    assert hits > 0
