"""GPU curvilinear state variant (state_kind 1: the (s, e_y, e_psi) state of the
paper's AutoRally model, Sec. VI-A, on the curvature of the centreline's
turning angles, Frenet kinematics) against the FP64 oracle.

  * K = 256, T = 50 on the ellipse track, from the centreline and from an
    off-centre start: every rollout cost and every trajectory state within
    1e-4 relative, V+ within the update bound;
  * ragged sizes (K not a multiple of the block, odd T) and the full-size
    K = 65536, T = 100 launch (sampled rollouts, V+);
  * the closed-loop step (Eq. 26) on the curvilinear state;
  * the shield (Alg. 1, modes 1 and 0) on near-edge curvilinear sequences and
    one whole Shield-MPPI update (rollouts, softmin, repair of V+, closed-loop
    step) against the oracle, repaired controls within V_REP unless a
    line-search decision differs between float32 and float64 (a flip);
  * smppi_cost_grad (full tape) against the oracle's dual-number gradient:
    J within S_REL, the gradient within G_REL on kink-free sequences;
  * the BFGS repair (mode 2) against the oracle's BFGS on
    near-edge curvilinear sequences (controls within V_REP unless a flip, at
    most 1/8), and a batch larger than the resident warps (warps take several
    sequences and reuse their H slice) bit-identical to a small batch on the
    sequences they share;
  * a track with two coinciding consecutive vertices (undefined curvature) is
    refused at smppi_create for the curvilinear state and accepted for the
    Cartesian one.
Tolerances: tests/gpu_helpers.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import (G_REL, S_REL, V_REP, X_REL, rel_err,  # noqa: E402
                                repair_compare, update_bound)


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def curv_problem(K, T, x0=(5.0, 0.0, 0.0, 0.0, 0.0, 0.0), **over):
    pr = I.single_problem(K=K, T=T, **over)
    pr.params["state_kind"] = 1
    pr.x0 = np.array(x0, np.float32)
    return pr


def gpu_step(S, pr, it=0, inst=0, traj=False):
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Sg, tr = ctl.step(x0, V, iter=it, instance=inst, want_S=True, want_traj=traj)
    st, bits = ctl.sync_status()
    assert st == S.OK, (st, bits)
    out = (Sg.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64),
           None if tr is None else tr.cpu().numpy().astype(np.float64))
    ctl.close()
    return out


def check_against_oracle(orc, pr, Sg, Vg, tr, ks, it=0, inst=0):
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, pr.x0, pr.V, it, inst, nthreads=8)
    _, om = orc.update(m, So, pr.V, it, inst)
    eps = orc.noise_block(m, it, inst, range(m.K))
    assert rel_err(Sg, So) <= S_REL
    ex = 0.0
    if tr is not None:
        for k in ks:
            _, to, _ = orc.rollout(m, pr.x0, pr.V, k=int(k), it=it, instance=inst)
            e = rel_err(tr[k], to)
            ex = max(ex, e)
            assert e <= X_REL, (k, e)
    tol = update_bound(So, eps, om, Vp, pr.V, pr.params["lam"])
    assert np.all(np.abs(Vg - Vp) <= tol)
    return rel_err(Sg, So), ex, np.abs(Vg - Vp).max()


@pytest.mark.parametrize("x0", [(5.0, 0.0, 0.0, 0.0, 0.0, 0.0), (6.0, 0.3, 0.2, 7.0, 1.2, 0.15)])
def test_curv_step_small_elementwise(S, orc, x0):
    pr = curv_problem(256, 50, x0)
    Sg, Vg, tr = gpu_step(S, pr, traj=True)
    es, ex, ev = check_against_oracle(orc, pr, Sg, Vg, tr, range(pr.K))
    print("curvilinear K=256 T=50 x0=%s: max rel S err %.2e, state %.2e, |V+ err| %.2e"
          % (x0, es, ex, ev))


@pytest.mark.parametrize("K,T", [(300, 37), (1, 1), (257, 2)])
def test_curv_step_ragged(S, orc, K, T):
    pr = curv_problem(K, T, (5.5, -0.1, 0.05, 30.0, -0.6, -0.1))
    Sg, Vg, tr = gpu_step(S, pr, it=3, inst=2, traj=True)
    check_against_oracle(orc, pr, Sg, Vg, tr, range(K), it=3, inst=2)


def test_curv_step_full_size(S, orc):
    pr = curv_problem(65536, 100)
    Sg, Vg, tr = gpu_step(S, pr, it=1, traj=True)
    ks = np.random.default_rng(0).choice(pr.K, 48, replace=False)
    es, ex, ev = check_against_oracle(orc, pr, Sg, Vg, tr, ks, it=1)
    print("curvilinear K=65536 T=100: max rel S err %.2e, state (48 sampled) %.2e, |V+ err| %.2e"
          % (es, ex, ev))


def test_curv_apply(S, orc):
    pr = curv_problem(64, 20, (6.0, 0.3, 0.2, 7.0, 1.2, 0.15))
    m = orc.Model(pr.params, pr.track)
    ctl = S.Controller(pr.params, pr.track)
    rng = np.random.default_rng(1)
    for n in range(5):
        V = rng.uniform(-0.4, 0.4, (pr.T, 2)).astype(np.float32)
        x0 = ctl.tensor(pr.x0)
        Vd = ctl.tensor(V)
        S.smppi_apply(ctl.h, x0, Vd, Vd, n, 3)
        assert ctl.sync_status()[0] == S.OK
        xo = orc.apply(m, pr.x0, V[0], n, 3)
        assert rel_err(x0.cpu().numpy(), xo) <= X_REL
        assert np.array_equal(Vd.cpu().numpy(), orc.shift(m, V).astype(np.float32))
    ctl.close()


def near_edge(n=16, T=40, seed=3):
    """Curvilinear starts near the track edge heading toward it, with smooth
    controls that steer further out (the shield's inputs)."""
    sb = I.near_edge_curvilinear(n, T, seed)
    return sb, sb.x0, sb.V


@pytest.mark.parametrize("mode", [1, 0])
def test_curv_repair_vs_oracle(S, orc, mode):
    pr, x0s, Vs = near_edge()
    if mode == 1:
        flips, worst = repair_compare(S, orc, pr.params, pr.track, x0s, Vs, 10)
        print("curvilinear repair (16 sequences, 10 Armijo iterations): %d flips, worst |dV| %.2e"
              % (flips, worst))
        assert worst <= V_REP and flips <= len(x0s) // 8
        return
    n = len(x0s)
    ctl = S.Controller(pr.params, pr.track, max_seq=n)
    Vout = torch.empty((n, pr.T, 2), device="cuda")
    S.smppi_repair(ctl.h, n, ctl.tensor(x0s), ctl.tensor(Vs), Vout, 1, 0, 1e-6)
    assert ctl.sync_status()[0] == S.OK
    m = orc.Model(pr.params, pr.track)
    for i in range(n):
        Vo = orc.repair(m, x0s[i], Vs[i], 1, mode=0, delta=1e-6)[0]
        assert np.max(np.abs(Vout[i].cpu().numpy() - Vo)) <= V_REP
    ctl.close()


@pytest.mark.parametrize("ey,ep", [(1.7, 0.25), (-1.6, -0.3), (0.0, 0.0)])
def test_curv_shield_update_vs_oracle(S, orc, ey, ep):
    # one whole Shield-MPPI update on the curvilinear state from a start near the
    # edge and heading out, against the oracle's mppi_step -> repair -> apply -> shift
    pr = curv_problem(512, 50, (6.0, 0.0, 0.0, 5.0, ey, ep))
    x0 = pr.x0
    V = np.tile(np.array([[0.0, 0.3]], np.float32), (pr.T, 1))
    it, inst = 3, 2
    ctl = S.Controller(pr.params, pr.track)
    xg, Vg, Vsg = ctl.tensor(x0), ctl.tensor(V), torch.empty((pr.T, 2), device="cuda")
    mer_g = torch.empty(11, dtype=torch.float64, device="cuda")
    S.smppi_shield_update(ctl.h, xg, Vg, Vsg, it, inst, 10, mer_g)
    st, bits = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), (st, bits)
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, x0, V, it, inst, nthreads=8)
    Vsafe, mer, ost, its = orc.repair(m, x0, Vp.astype(np.float32), 10)
    x1 = orc.apply(m, x0, Vsafe[0], it, inst)
    print("curvilinear e_y %.1f: oracle repair iterations %d, merit %.4g -> %.4g"
          % (ey, its, mer[0], mer[its]))
    _, om = orc.update(m, So, V, it, inst)
    eps = orc.noise_block(m, it, inst, range(m.K))
    tol = update_bound(So, eps, om, Vp, V, pr.params["lam"])
    tol_sh = np.concatenate([tol[1:], tol[-1:]])
    assert np.all(np.abs(Vg.cpu().numpy() - orc.shift(m, Vp)) <= tol_sh)
    assert np.max(np.abs(Vsg.cpu().numpy() - Vsafe)) <= V_REP
    assert rel_err(xg.cpu().numpy(), x1) <= X_REL
    assert mer_g.cpu().numpy()[0] == pytest.approx(mer[0], rel=S_REL, abs=1e-2)
    ctl.close()


def test_curv_shield_device_host_graph_agree(S):
    pr = curv_problem(256, 30, (6.0, 0.0, 0.0, 5.0, 1.5, 0.2))
    ctl = S.Controller(pr.params, pr.track)
    ref = None
    for how in ("device", "host", "graph"):
        x0 = ctl.tensor(pr.x0)
        V = ctl.tensor(pr.V)
        Vs = torch.empty_like(V)
        if how == "device":
            for n in range(3):
                S.smppi_shield_update(ctl.h, x0, V, Vs, n, 0, 5)
            out = (x0.cpu().numpy(), V.cpu().numpy(), Vs.cpu().numpy())
        elif how == "host":
            hx, hV = pr.x0.copy(), pr.V.copy()
            hVs = np.empty_like(hV)
            for n in range(3):
                S.smppi_shield_update(ctl.h, hx.ctypes.data, hV.ctypes.data, hVs.ctypes.data, n, 0,
                                      5, None, True)
            out = (hx, hV, hVs)
        else:
            S.smppi_shield_loop(ctl.h, x0, V, Vs, 0, 0, 5, 3)
            out = (x0.cpu().numpy(), V.cpu().numpy(), Vs.cpu().numpy())
        assert ctl.sync_status()[0] in (S.OK, S.ERR_STALLED)
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b), how
    ctl.close()


@pytest.mark.parametrize("w_run,w_cbf", [(1.0, 1.0), (0.0, 1.0), (1.0, 0.0)])
def test_curv_cost_grad_vs_oracle(S, orc, w_run, w_cbf):
    # J within S_REL and the adjoint gradient within G_REL (relative l2) of the
    # oracle's dual-number gradient on sequences with no max(0, .) kink within 1e-3
    pr, x0s, Vs = near_edge(n=24, T=40, seed=7)
    n = len(x0s)
    ctl = S.Controller(pr.params, pr.track, max_seq=n)
    J = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, pr.T, 2), device="cuda")
    S.smppi_cost_grad(ctl.h, n, ctl.tensor(x0s), ctl.tensor(Vs), pr.T, w_run, w_cbf, 0, J, g)
    assert ctl.sync_status()[0] == S.OK
    J, g = J.cpu().numpy(), g.cpu().numpy().astype(np.float64)
    ctl.close()
    m = orc.Model(pr.params, pr.track)
    a1 = 1 - float(np.float32(pr.params["alpha"]))
    w2 = float(np.float32(pr.params["half_width"])) ** 2
    clean, worst = 0, 0.0
    for i in range(n):
        Jo, go = orc.cost_grad(m, x0s[i], Vs[i], None, w_run, w_cbf)
        assert abs(J[i] - Jo) <= S_REL * (abs(Jo) + 1), (i, J[i], Jo)
        _, traj, _ = orc.rollout(m, x0s[i], Vs[i], noisy=False)
        h = w2 - traj[:, 4] ** 2
        if w_cbf != 0.0 and np.any(np.abs(a1 * h[:-1] - h[1:]) < 1e-3):
            continue
        e = np.linalg.norm(g[i] - go) / max(np.linalg.norm(go), 1e-12)
        worst = max(worst, e)
        clean += 1
    print("curvilinear cost_grad (%g, %g): %d kink-free of %d, worst rel l2 %.2e"
          % (w_run, w_cbf, clean, n, worst))
    assert clean >= 8 and worst <= G_REL


def test_curv_bfgs_vs_oracle(S, orc):
    pr, x0s, Vs = near_edge(n=64, T=40, seed=7)
    flips, worst = repair_compare(S, orc, pr.params, pr.track, x0s, Vs, 10, mode=2)
    print("curvilinear BFGS repair (64 sequences, 10 iterations): %d flips, worst |dV| %.2e"
          % (flips, worst))
    assert worst <= V_REP and flips <= len(x0s) // 8


def _bfgs_run(S, ctl, x0, V, n, n_iters):
    Vout = torch.empty((n, ctl.T, 2), device="cuda")
    mer = torch.empty((n, n_iters + 1), dtype=torch.float64, device="cuda")
    its = torch.empty(n, dtype=torch.int32, device="cuda")
    S.smppi_repair(ctl.h, n, x0[:n], V[:n], Vout, n_iters, 2, 0.0, mer, its)
    st, _ = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED)
    return Vout.cpu().numpy(), mer.cpu().numpy(), its.cpu().numpy()


def test_curv_bfgs_independent_of_batch(S):
    n = 8192          # more than the resident warps of the T = 40 launch
    pr, x0s, Vs = near_edge(n=n, T=40, seed=11)
    ctl = S.Controller(pr.params, pr.track, max_seq=n)
    x0, V = ctl.tensor(x0s), ctl.tensor(Vs)
    big = _bfgs_run(S, ctl, x0, V, n, 10)
    small = _bfgs_run(S, ctl, x0, V, 256, 10)
    ctl.close()
    for a, b in zip(big, small):
        assert np.array_equal(a[:256], b)
    mer = big[1]
    assert np.all(mer[:, -1] <= mer[:, 0])
    print("curvilinear BFGS, %d sequences: safe after %d of %d unsafe"
          % (n, int(((mer[:, 0] > 0) & (mer[:, -1] == 0)).sum()), int((mer[:, 0] > 0).sum())))


def test_curv_degenerate_track_refused(S):
    pr = curv_problem(64, 20)
    tr = pr.track.copy()
    tr[5] = tr[4]
    with pytest.raises(S.SmppiError) as ei:
        S.Controller(pr.params, tr)
    assert ei.value.status == S.ERR_ARG and "vertices" in str(ei.value)
    p0 = dict(pr.params)
    p0["state_kind"] = 0
    ctl = S.Controller(p0, tr)
    x0, V = ctl.tensor(I.single_problem(K=64, T=20).x0), ctl.tensor(pr.V)
    ctl.step(x0, V)
    assert ctl.sync_status()[0] == S.OK
    ctl.close()
