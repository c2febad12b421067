"""GPU curvilinear state variant (state_kind 1: the (s, e_y, e_psi) state of the
paper's AutoRally model, Sec. VI-A; readings c28, c29) against the FP64 oracle.

  * K = 256, T = 50 on the ellipse track, from the centreline and from an
    off-centre start: every rollout cost and every trajectory state within
    1e-4 relative, V+ within the update bound;
  * ragged sizes (K not a multiple of the block, odd T) and the full-size
    K = 65536, T = 100 launch (sampled rollouts, V+);
  * the closed-loop step (Eq. 26) on the curvilinear state;
  * the repair, adjoint, shield and batch entry points refuse state_kind 1.
Tolerances: tests/gpu_helpers.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import S_REL, X_REL, rel_err, update_bound  # noqa: E402


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


def test_curv_refused_entry_points(S):
    pr = curv_problem(64, 20)
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    with pytest.raises(RuntimeError):
        S.smppi_repair(ctl.h, 1, x0, V, Vs, 5, 1)
    with pytest.raises(RuntimeError):
        S.smppi_shield_update(ctl.h, x0, V, Vs, 0, 0, 5)
    ctl.close()
