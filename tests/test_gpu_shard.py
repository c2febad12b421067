"""Rollout sharding on the GPU: smppi_step_partial over slices of the K
rollouts, then smppi_merge_partials (Eq. 10-11 over a partition of the
rollouts, log-sum-exp merge of the per-slice min-shifted sums).

  * one slice holding all K rollouts, merged, gives smppi_step's V+ bit for bit
    (same kernels, the merge's rescaling factor is exactly 1);
  * 2, 3 and 8 uneven slices (boundaries off the 256-rollout blocks) give
    smppi_step's V+ to float32 rounding of the block sums (1e-6), at the
    K = 65536, T = 100 size that bench.py times;
  * each GPU slice partial matches the oracle's partial of the same slice from
    the oracle's costs (m_g within the cost tolerance, and the slice's own
    update within the end-to-end update bound), and the merged V+ matches the
    oracle's merge of its partials within that bound.
Tolerances: tests/gpu_helpers.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import S_REL, V_UPD, update_bound  # noqa: E402


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _sharded(S, ctl, x0, V, bounds, it, inst=0):
    T = ctl.T
    parts = torch.empty((len(bounds) - 1, 2 * T + 2), dtype=torch.float64, device="cuda")
    for g in range(len(bounds) - 1):
        S.smppi_step_partial(ctl.h, x0, V, it, inst, int(bounds[g]), int(bounds[g + 1]), parts[g])
    Vm = V.clone()
    S.smppi_merge_partials(ctl.h, len(bounds) - 1, parts, Vm)
    return parts, Vm


@pytest.mark.parametrize("K,T", [(65536, 100), (1000, 51)])
def test_one_slice_is_the_step(S, K, T):
    pr = I.throughput_problem(K, T)
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    _, Vm = _sharded(S, ctl, x0, V, [0, K], 1)
    Vs = V.clone()
    S.smppi_step(ctl.h, x0, Vs, 1, 0, None, None)
    torch.cuda.synchronize()
    assert ctl.sync_status()[0] == S.OK
    assert torch.equal(Vm, Vs)
    ctl.close()


def test_slices_merge_to_the_step(S):
    K, T = 65536, 100
    pr = I.throughput_problem(K, T)
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    Vs = V.clone()
    S.smppi_step(ctl.h, x0, Vs, 2, 0, None, None)
    for bounds in ([0, 32768, K], [0, 20001, 40000, K], list(np.linspace(0, K, 9).astype(int) +
                                                              np.array([0, 7, 3, 100, 5, 1, 9, 77, 0]))):
        _, Vm = _sharded(S, ctl, x0, V, bounds, 2)
        torch.cuda.synchronize()
        e = (Vm - Vs).abs().max().item()
        print("%d slices: max |V+ (merged) - V+ (one launch)| = %.2e" % (len(bounds) - 1, e))
        assert e <= 1e-6
    assert ctl.sync_status()[0] == S.OK
    ctl.close()


def test_partials_and_merge_vs_oracle(S, orc):
    K, T = 4096, 64
    pr = I.throughput_problem(K, T)
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    bounds = [0, 1000, 2500, K]
    parts, Vm = _sharded(S, ctl, x0, V, bounds, 7, 3)
    torch.cuda.synchronize()
    assert ctl.sync_status()[0] == S.OK
    parts, Vm = parts.cpu().numpy(), Vm.cpu().numpy().astype(np.float64)
    m = orc.Model(pr.params, pr.track)
    So, Vp = orc.mppi_step(m, pr.x0, pr.V, 7, 3, nthreads=16)
    lam = pr.params["lam"]
    po = []
    for g in range(3):
        lo, hi = bounds[g], bounds[g + 1]
        pg = orc.partial(m, So[lo:hi], lo, 7, 3)
        po.append(pg)
        assert abs(parts[g][0] - pg[0]) <= S_REL * (abs(pg[0]) + 1.0)
        # the slice's own update V + A_g / eta_g, GPU against oracle, within the
        # end-to-end update bound of that slice's costs
        Vg_gpu = pr.V + (parts[g][2:] / parts[g][1]).reshape(T, 2)
        Vg_orc = pr.V + (pg[2:] / pg[1]).reshape(T, 2)
        w = np.exp(-(So[lo:hi] - pg[0]) / lam)
        w /= w.sum()
        eps = orc.noise_block(m, 7, 3, range(lo, hi))
        tol = update_bound(So[lo:hi], eps, w, Vg_orc, pr.V, lam)
        assert np.all(np.abs(Vg_gpu - Vg_orc) <= tol), g
    Vmo = orc.merge(m, np.stack(po), pr.V)
    assert np.max(np.abs(Vmo - Vp)) < 1e-12
    _, om = orc.update(m, So, pr.V, 7, 3)
    eps = orc.noise_block(m, 7, 3, range(K))
    tol = update_bound(So, eps, om, Vp, pr.V, lam)
    e = np.abs(Vm - Vp)
    assert np.all(e <= tol)
    print("3 slices vs the oracle: max |V+ err| %.2e (bound min %.2e)" % (e.max(), tol.min()))
    assert e.max() <= V_UPD
    ctl.close()


def test_partial_argument_checks(S):
    pr = I.throughput_problem(1024, 20)
    ctl = S.Controller(pr.params, pr.track)
    x0, V = ctl.tensor(pr.x0), ctl.tensor(pr.V)
    part = torch.empty(42, dtype=torch.float64, device="cuda")
    for lo, hi in ((0, 0), (5, 4), (-1, 10), (0, 1025)):
        with pytest.raises(S.SmppiError) as err:
            S.smppi_step_partial(ctl.h, x0, V, 0, 0, lo, hi, part)
        assert err.value.status == S.ERR_ARG
    for n in (0, 1025):
        with pytest.raises(S.SmppiError) as err:
            S.smppi_merge_partials(ctl.h, n, part, V)
        assert err.value.status == S.ERR_ARG
    ctl.close()
