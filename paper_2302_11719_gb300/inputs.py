"""Seeded synthetic inputs for the Shield-MPPI hot path.

This module only produces numbers that go INTO a control update: parameter
values, centreline tables, initial states and initial control sequences.  It
holds none of the method's arithmetic (no dynamics, no costs, no noise of the
method, no weights), so the CUDA path and the CPU oracle can both take their
inputs from here without sharing any of the computation they are checked on.

The paper (arXiv 2302.11719, Sec. VI) runs on the AutoRally track and
simulator, which are not available; elliptical tracks of constant half-width
stand in for them.  Values of the model and cost follow the workload
definitions: 6-state single-track car, m = 21.7 kg, Iz = 1.12 kg m^2,
lf = 0.34 m, lr = 0.23 m, tyre B = 4, C = 1.5, rear force 60 N per unit
throttle, Euler dt = 0.02 s, Sigma = diag(0.15^2, 0.3^2), lambda = 1,
alpha = 0.3 (the paper's beta), C = 1000, cost 2 (v_x - 8)^2 + 100 e_y^2 / w^2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Parameter values of the single-problem workloads (names follow the paper:
# lambda = temperature, alpha = class-kappa rate (paper's beta), C_cbf = C).
DEFAULT_PARAMS = dict(
    m=21.7, Iz=1.12, lf=0.34, lr=0.23,
    B=4.0, Ct=1.5, g=9.81, fx_gain=60.0,
    dt=0.02,
    sigma=(0.15, 0.3),
    lam=1.0, gamma=1.0,
    K=256, T=50, N_r=50,
    alpha=0.3, C_cbf=1000.0,
    q_v=2.0, v_target=8.0, q_d=100.0, C_obs=0.0,
    u_min=(-0.5, -1.0), u_max=(0.5, 1.0),
    half_width=2.0,
    dist_sigma=(0.3, 0.3),
    ls_s0=0.1, ls_c=1e-4, ls_max_halvings=20,
    seed=0,
)

N_TRACK = 1024


@dataclasses.dataclass
class Problem:
    """One control problem: parameters, centreline, state and nominal controls."""
    params: dict
    track: np.ndarray      # (n_track, 2) float32, closed polyline, counter-clockwise
    x0: np.ndarray         # (6,) float32: (v_x, v_y, r, X, Y, psi)
    V: np.ndarray          # (T, 2) float32: (steer, throttle)

    @property
    def K(self) -> int:
        return int(self.params["K"])

    @property
    def T(self) -> int:
        return int(self.params["T"])


def make_params(**over) -> dict:
    p = dict(DEFAULT_PARAMS)
    p.update(over)
    if "gamma" not in over and "lam" in over:
        p["gamma"] = p["lam"]
    if "N_r" not in over:
        p["N_r"] = p["T"]
    return p


def ellipse_track(a: float, b: float, n: int = N_TRACK) -> np.ndarray:
    """Centreline points E(theta_i) = (a cos theta_i, b sin theta_i), theta_i = 2 pi i / n."""
    th = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n
    return np.stack([a * np.cos(th), b * np.sin(th)], axis=1).astype(np.float32)


def centreline_start(a: float, b: float, vx: float) -> np.ndarray:
    """State on the centreline at theta = 0, heading along the CCW tangent."""
    return np.array([vx, 0.0, 0.0, a, 0.0, math.pi / 2], dtype=np.float32)


def single_problem(K: int = 256, T: int = 50, a: float = 20.0, b: float = 12.0,
                   w: float = 2.0, vx: float = 5.0, **over) -> Problem:
    """The single-problem workload: ellipse a x b, half-width w, V = 0."""
    p = make_params(K=K, T=T, half_width=w, **over)
    return Problem(params=p, track=ellipse_track(a, b), x0=centreline_start(a, b, vx),
                   V=np.zeros((T, 2), dtype=np.float32))


def single_step_small() -> Problem:
    """K = 256, T = 50 step followed by 10 repair steps."""
    return single_problem(K=256, T=50)


def closed_loop_plain() -> Problem:
    """K = 1024, T = 60 closed loop without the shield (no repair, no CBF cost)."""
    return single_problem(K=1024, T=60, C_cbf=0.0)


def throughput_problem(K: int, T: int) -> Problem:
    """Rollout-throughput sweep point (K, T) on the single-problem model and track."""
    return single_problem(K=K, T=T)


def _tangent_normal(a: float, b: float, th: np.ndarray):
    tx, ty = -a * np.sin(th), b * np.cos(th)
    n = np.hypot(tx, ty)
    tx, ty = tx / n, ty / n
    return tx, ty, -ty, tx   # unit tangent (CCW) and left normal


@dataclasses.dataclass
class SequenceBatch:
    """Many independent (x0, V) pairs on one track (gradient / repair workload)."""
    params: dict
    track: np.ndarray
    x0: np.ndarray        # (n_seq, 6) float32
    V: np.ndarray         # (n_seq, T, 2) float32
    side: np.ndarray      # (n_seq,) +1 = offset to the left of the centreline, -1 right

    @property
    def T(self) -> int:
        return int(self.params["T"])


def near_boundary_sequences(n_seq: int = 8192, T: int = 100, seed: int = 0,
                            a: float = 20.0, b: float = 12.0, w: float = 2.0) -> SequenceBatch:
    """Control sequences of the kind an MPPI update returns, perturbed toward the boundary.

    theta0 ~ U[0, 2 pi), lateral offset d0 ~ U[1.5, 1.95] m on a random side,
    heading = tangent + 0.1 rad toward that side, v_x ~ U[5, 8] m/s.  Steering
    follows the local centreline curvature (kinematic steer (lf + lr) kappa),
    plus a smooth (AR(1), rho = 0.9) Gaussian perturbation of std 0.05 and a
    0.05 rad bias toward the offset side; throttle is a smooth perturbation
    around 0.2.  All values are clamped to the control box.
    """
    rng = np.random.default_rng([seed, 3])
    p = make_params(T=T, N_r=T, half_width=w)
    th = rng.uniform(0.0, 2 * np.pi, n_seq)
    side = np.where(rng.uniform(size=n_seq) < 0.5, 1.0, -1.0)
    d0 = rng.uniform(1.5, 1.95, n_seq)
    vx = rng.uniform(5.0, 8.0, n_seq)
    tx, ty, nx, ny = _tangent_normal(a, b, th)
    X = a * np.cos(th) + side * d0 * nx
    Y = b * np.sin(th) + side * d0 * ny
    psi = np.arctan2(ty, tx) + side * 0.1
    x0 = np.stack([vx, np.zeros(n_seq), np.zeros(n_seq), X, Y, psi], axis=1).astype(np.float32)
    # curvature of the ellipse along the path travelled at v_x (arc length ~ v_x t dt)
    L = p["lf"] + p["lr"]
    t = np.arange(T)
    speed_arc = vx[:, None] * p["dt"] * t[None, :]
    # d theta / ds = 1 / |E'(theta)|
    dth = speed_arc / np.hypot(a * np.sin(th), b * np.cos(th))[:, None]
    thp = th[:, None] + dth
    kappa = a * b / np.power(a * a * np.sin(thp) ** 2 + b * b * np.cos(thp) ** 2, 1.5)
    steer = np.arctan(L * kappa)

    def ar1(scale):
        e = rng.normal(0.0, 1.0, (n_seq, T))
        out = np.empty_like(e)
        acc = e[:, 0]
        out[:, 0] = acc
        rho = 0.9
        for j in range(1, T):
            acc = rho * acc + math.sqrt(1 - rho * rho) * e[:, j]
            out[:, j] = acc
        return scale * out

    steer = steer + ar1(0.05) + 0.05 * side[:, None]
    thr = 0.2 + ar1(0.2)
    V = np.stack([np.clip(steer, -0.5, 0.5), np.clip(thr, -1.0, 1.0)], axis=2).astype(np.float32)
    return SequenceBatch(params=p, track=ellipse_track(a, b), x0=x0, V=V, side=side)


def near_edge_curvilinear(n_seq: int = 16, T: int = 40, seed: int = 3) -> SequenceBatch:
    """Curvilinear-state starts (state_kind 1) near the edge of the single-problem
    track, heading toward it, with smooth controls that steer further out.

    Sequence i takes side +1 (left) for even i, -1 for odd i; x0 = (v_x, 0, 0,
    s, side e_y, side 0.08) with v_x ~ U[5, 8] m/s, s ~ U[0, 60] m and
    e_y ~ U[1.4, 1.8] m (half-width 2); steering side 0.06 + N(0, 0.04^2) and
    throttle 0.2 + N(0, 0.2^2) per step, independent, clipped to
    [-0.45, 0.45] x [-0.9, 0.9].  The draws are taken sequence by sequence
    from default_rng(seed).
    """
    pr = single_problem(K=1, T=T)
    p = dict(pr.params)
    p["state_kind"] = 1
    rng = np.random.default_rng(seed)
    x0s, Vs, sides = [], [], []
    for i in range(n_seq):
        side = 1.0 if i % 2 == 0 else -1.0
        x0s.append([rng.uniform(5, 8), 0.0, 0.0, rng.uniform(0, 60), side * rng.uniform(1.4, 1.8),
                    side * 0.08])
        steer = side * 0.06 + 0.04 * rng.standard_normal(T)
        thr = 0.2 + 0.2 * rng.standard_normal(T)
        Vs.append(np.clip(np.stack([steer, thr], 1), [-0.45, -0.9], [0.45, 0.9]))
        sides.append(side)
    return SequenceBatch(params=p, track=pr.track, x0=np.array(x0s, np.float32),
                         V=np.array(Vs, np.float32), side=np.array(sides))


@dataclasses.dataclass
class InstanceBatch:
    """Independent control problems with uneven K and T (batched workload)."""
    params: list          # per-instance parameter dicts
    tracks: np.ndarray    # (n_inst, n_track, 2) float32
    x0: np.ndarray        # (n_inst, 6) float32
    K: np.ndarray         # (n_inst,) int
    T: np.ndarray         # (n_inst,) int
    a: np.ndarray
    b: np.ndarray
    w: np.ndarray


# Closed-loop stress setting of the controller comparison: a high target speed,
# weak centring and strong disturbances on narrow tracks (w in [1, 1.5] m), so
# that the three controllers' CBF-violation rates differ.
HARSH = dict(v_target=14.0, q_d=10.0, dist_sigma=(0.6, 0.6))


def uneven_instances(n_inst: int = 512, seed: int = 0, K_lo: int = 64, K_hi: int = 16384,
                     T_lo: int = 20, T_hi: int = 150, w_lo: float = 1.5, w_hi: float = 3.0,
                     **over) -> InstanceBatch:
    """K log-uniform in [K_lo, K_hi], T uniform in {T_lo..T_hi}, a, b ~ U[10, 40] m,
    w ~ U[w_lo, w_hi] m (default [1.5, 3]), resampled until min(a,b)^2 / max(a,b) > 2 w
    (no cusp on the inner boundary); x0 on the centreline at theta = 0 with
    v_x ~ U[4, 6] m/s.  over: parameter overrides shared by all problems."""
    rng = np.random.default_rng([seed, 4])
    Ks = np.rint(np.exp(rng.uniform(math.log(K_lo), math.log(K_hi), n_inst))).astype(np.int64)
    Ts = rng.integers(T_lo, T_hi + 1, n_inst)
    a = np.empty(n_inst); b = np.empty(n_inst); w = np.empty(n_inst)
    for i in range(n_inst):
        while True:
            ai, bi, wi = rng.uniform(10, 40), rng.uniform(10, 40), rng.uniform(w_lo, w_hi)
            if min(ai, bi) ** 2 / max(ai, bi) > 2 * wi:
                break
        a[i], b[i], w[i] = ai, bi, wi
    vx = rng.uniform(4.0, 6.0, n_inst)
    tracks = np.stack([ellipse_track(a[i], b[i]) for i in range(n_inst)])
    x0 = np.stack([centreline_start(a[i], b[i], vx[i]) for i in range(n_inst)])
    params = [make_params(K=int(Ks[i]), T=int(Ts[i]), half_width=float(w[i]), seed=seed, **over)
              for i in range(n_inst)]
    return InstanceBatch(params=params, tracks=tracks, x0=x0, K=Ks, T=Ts, a=a, b=b, w=w)
