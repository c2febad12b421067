"""Parity at the workload sizes of the measurements, with the errors printed.

  * the MPPI iteration at K = 65536 and 262144, T = 100: V+ against the
    oracle's V+ (the end-to-end update bound, and the maximum error printed);
  * the whole Shield-MPPI update at the same sizes through the launch pair
    bench.py times (rollouts that also write block partials, then one block
    that merges them into V+, runs the shield and takes the closed-loop step):
    the warm start shift(V+) within the update bound, V_safe within the repair
    tolerance plus that bound, the executed step within 1e-4 relative;
  * the shield on 8192 near-boundary sequences, T = 100, 20 iterations, run in
    the launch shape of that size (one block per sequence for the gradient
    repair, one warp per sequence for BFGS), compared with the oracle's repair
    on every 32nd sequence: flips (line-search decisions taken differently in
    float32 and float64) counted and printed, the other sequences within 1e-4;
  * the batch of 512 uneven problems (K log-uniform in [64, 16384], T in
    [20, 150]): 20 closed-loop updates in one persistent launch each, 16
    problems spread over the K and T range resynced to the oracle at every
    update and compared: V+ within the update bound; V_safe within 1e-4 plus
    the bound of the V+ it starts from (else a flip); the executed closed-loop
    step, from the control the GPU executed, within 1e-4 relative.
The oracle runs on host threads (its C routines release the interpreter lock).
Tolerances: tests/gpu_helpers.py.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import S_REL, V_REP, V_UPD, X_REL, rel_err, update_bound  # noqa: E402

N_THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _bound_top(orc, m, So, V, Vp, it, inst, lam):
    """The update bound from the weights that carry all but 1e-12 of the mass."""
    _, om = orc.update(m, So, V, it, inst)
    order = np.argsort(-om)
    n = int(np.searchsorted(np.cumsum(om[order]), 1 - 1e-12)) + 1
    top = order[:max(n, 8)]
    eps = orc.noise_block(m, it, inst, [int(k) for k in top])
    return update_bound(So[top], eps, om[top], Vp, V, lam)


@pytest.mark.parametrize("K", [65536, 262144])
def test_update_error_full_size(S, orc, K):
    pr = I.throughput_problem(K, 100)
    ctl = S.Controller(pr.params, pr.track)
    V = ctl.tensor(pr.V)
    Sg, _ = ctl.step(ctl.tensor(pr.x0), V, iter=1, want_S=True)
    assert ctl.sync_status()[0] == S.OK
    Sg, Vg = Sg.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    ctl.close()
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, pr.x0, pr.V, 1, 0, nthreads=N_THREADS)
    es = rel_err(Sg, So)
    assert es <= S_REL
    tol = _bound_top(orc, m, So, pr.V, Vp, 1, 0, pr.params["lam"])
    e = np.abs(Vg - Vp)
    print("K=%d T=100: max rel S err %.2e, max |V+ err| %.2e (gate %.0e; update bound "
          "here %.2e..%.2e)" % (K, es, e.max(), V_UPD, tol.min(), tol.max()))
    assert np.all(e <= tol)
    assert e.max() <= V_UPD


@pytest.mark.parametrize("K", [65536, 262144])
def test_shield_update_full_size(S, orc, K):
    pr = I.throughput_problem(K, 100)
    it, inst = 1, 0
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, 10)
    st, _ = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), st
    Vg, Vsg = V.cpu().numpy().astype(np.float64), Vs.cpu().numpy()
    xg = x0.cpu().numpy()
    ctl.close()
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, pr.x0, pr.V, it, inst, nthreads=N_THREADS)
    tol = _bound_top(orc, m, So, pr.V, Vp, it, inst, pr.params["lam"])
    tol_sh = np.concatenate([tol[1:], tol[-1:]])
    e_sh = np.abs(Vg - orc.shift(m, Vp))
    Vso, mer, _, its = orc.repair(m, pr.x0, Vp.astype(np.float32), 10)
    e_s = np.abs(Vsg.astype(np.float64) - Vso)
    x1 = orc.apply(m, pr.x0, Vsg[0], it, inst)
    ex = rel_err(xg, x1)
    print("shield update K=%d T=100: max |shift(V+) err| %.2e (bound %.2e..%.2e), "
          "max |V_safe err| %.2e (oracle repair iterations %d), rel next-state err %.2e"
          % (K, e_sh.max(), tol.min(), tol.max(), e_s.max(), its, ex))
    assert np.all(e_sh <= tol_sh) and e_sh.max() <= V_UPD
    assert np.all(e_s <= V_REP + tol)
    assert ex <= X_REL


@pytest.mark.parametrize("T,K", [(1, 1 << 19), (2, 1 << 19), (51, 65536), (255, 16384),
                                 (256, 16384), (511, 8192), (512, 8192)])
def test_shield_update_horizons(S, orc, T, K):
    # the merge of the block partials at horizons from 1 to SMPPI_MAX_T (one
    # control per thread up to 2T = 256, several beyond) and from 32 to 2048
    # rollout blocks, against the oracle's V+ (the warm start shift(V+) within the
    # update bound), and V_safe = V+ where no repair ran
    pr = I.throughput_problem(K, T)
    it, inst = 2, 1
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = torch.empty_like(V)
    mer = torch.empty(11, dtype=torch.float64, device="cuda")
    S.smppi_shield_update(ctl.h, x0, V, Vs, it, inst, 10, mer)
    st, _ = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), st
    Vg, Vsg = V.cpu().numpy().astype(np.float64), Vs.cpu().numpy().astype(np.float64)
    ctl.close()
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, pr.x0, pr.V, it, inst, nthreads=N_THREADS)
    tol = _bound_top(orc, m, So, pr.V, Vp, it, inst, pr.params["lam"])
    tol_sh = np.concatenate([tol[1:], tol[-1:]])
    e_sh = np.abs(Vg - orc.shift(m, Vp))
    print("shield update K=%d T=%d: max |shift(V+) err| %.2e (bound %.2e..%.2e)"
          % (K, T, e_sh.max(), tol.min(), tol.max()))
    assert np.all(e_sh <= tol_sh) and e_sh.max() <= V_UPD
    if mer.cpu().numpy()[0] == 0.0:      # V+ already safe: V_safe is V+ itself
        assert np.all(np.abs(Vsg - Vp) <= tol)


def _repair_sample(S, orc, mode):
    sb = I.near_boundary_sequences(8192, 100, seed=0)
    n = sb.x0.shape[0]
    ctl = S.Controller(sb.params, sb.track, max_seq=n, checkpoint=10)
    Vout = torch.empty((n, 100, 2), device="cuda")
    its = torch.empty(n, dtype=torch.int32, device="cuda")
    S.smppi_repair(ctl.h, n, ctl.tensor(sb.x0), ctl.tensor(sb.V), Vout, 20, mode, 0.0, None, its)
    st, _ = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), st
    Vout, its = Vout.cpu().numpy(), its.cpu().numpy()
    ctl.close()
    m = orc.Model(sb.params, sb.track)
    idx = list(range(0, n, 32))

    def one(i):
        Vo, _, _, io = orc.repair(m, sb.x0[i], sb.V[i], 20, mode=mode)
        return i, Vo, io

    with cf.ThreadPoolExecutor(N_THREADS) as ex:
        res = list(ex.map(one, idx))
    flips, worst = 0, 0.0
    for i, Vo, io in res:
        e = np.max(np.abs(Vout[i] - Vo))
        if io != its[i] or e > V_REP:
            flips += 1
        else:
            worst = max(worst, e)
    return flips, len(idx), worst


@pytest.mark.parametrize("mode,name", [(1, "gradient + Armijo"), (2, "BFGS")])
def test_repair_8192_sampled(S, orc, mode, name):
    flips, n, worst = _repair_sample(S, orc, mode)
    print("8192 near-boundary sequences, %s repair, 20 iterations: %d flips in %d sampled, "
          "worst |V_safe err| of the others %.2e" % (name, flips, n, worst))
    assert worst <= V_REP and flips <= n // 8


def test_batch_512_spot_check(S, orc):
    ib = I.uneven_instances(512, seed=0)
    bt = S.Batch(ib, block_rollouts=0)
    B = bt.B
    # 16 problems spread over the sizes: the extremes of K and T, then by K T
    kt = ib.K * ib.T
    pick = {int(np.argmax(ib.K)), int(np.argmin(ib.K)), int(np.argmax(ib.T)), int(np.argmin(ib.T))}
    for i in np.argsort(kt)[np.linspace(0, B - 1, 16).astype(int)]:
        if len(pick) < 16:
            pick.add(int(i))
    pick = sorted(pick)
    models = {i: orc.Model(ib.params[i], ib.tracks[i]) for i in pick}
    xs = {i: ib.x0[i].astype(np.float64) for i in pick}
    Vs = {i: np.zeros((bt.T[i], 2)) for i in pick}
    flips = compared = 0
    worst_V = worst_x = 0.0

    def oracle_update(i, n):
        m = models[i]
        x32, V32 = xs[i].astype(np.float32), Vs[i].astype(np.float32)
        So, Vp = orc.mppi_step(m, x32, V32, n, i, nthreads=1)
        tol = _bound_top(orc, m, So, V32, Vp, n, i, ib.params[i]["lam"])
        Vso = orc.repair(m, x32, Vp.astype(np.float32), 10)[0]
        return i, Vp, tol, Vso, orc.apply(m, x32, Vso[0], n, i), orc.shift(m, Vp)

    with cf.ThreadPoolExecutor(N_THREADS) as ex:
        for n in range(20):
            x_all = bt.x0.cpu().numpy()
            V_all = bt.V.cpu().numpy()
            for i in pick:              # oracle -> GPU for the checked problems
                x_all[i] = xs[i]
                V_all[bt.V_off[i]:bt.V_off[i] + bt.T[i]] = Vs[i]
            bt.x0.copy_(torch.as_tensor(x_all))
            bt.V.copy_(torch.as_tensor(V_all))
            S.smppi_batch_step(bt.b, bt.x0, bt.V, bt.V_safe, n, 10)
            st, bits = S.smppi_batch_sync_status(bt.b)
            assert st in (S.OK, S.ERR_STALLED), (st, bits)
            Vg, Vsg, xg = bt.split(bt.V), bt.split(bt.V_safe), bt.x0.cpu().numpy()
            for i, Vp, tol, Vso, x1, Vsh in ex.map(lambda i: oracle_update(i, n), pick):
                tol_sh = np.concatenate([tol[1:], tol[-1:]])
                eV = np.abs(Vg[i] - Vsh)
                assert np.all(eV <= tol_sh), (n, i, eV.max())
                worst_V = max(worst_V, eV.max())
                compared += 1
                # V_safe starts from a V+ that may differ by the update bound: the repair
                # tolerance is added to it; beyond that a line-search decision differs
                if np.any(np.abs(Vsg[i] - Vso) > V_REP + tol):
                    flips += 1
                # the executed step, from the control the GPU executed
                x1g = orc.apply(models[i], xs[i].astype(np.float32), Vsg[i][0], n, i)
                ex_ = rel_err(xg[i], x1g)
                assert ex_ <= X_REL, (n, i, ex_)
                worst_x = max(worst_x, ex_)
                xs[i], Vs[i] = x1, Vsh
    rb, grid = S.smppi_batch_config(bt.b)
    bt.close()
    print("batch of 512 (autotuned %d rollouts per item, grid %d): %d problem-updates compared, "
          "max |V err| %.2e, max rel next-state err %.2e, %d repair flips"
          % (rb, grid, compared, worst_V, worst_x, flips))
    assert flips <= compared // 16
