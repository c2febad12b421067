"""The shield's block-parallel adjoint gradients (the block repair of the
Cartesian model and that of the curvilinear state) against the oracle's
dual-number gradient of the merit (running-cost weight 0, CBF weight 1).

One fixed-step iteration of smppi_repair (mode 0: V_out = clamp(V - delta G))
runs per sequence, with delta chosen so that delta max|G| = 0.02 (float32
rounding of V then limits the recovered gradient to about 4e-4 relative).  The
gradient is read back as (V - V_out) / delta on the components the box does not
clip and compared within G_REL relative l2 on sequences with no max(0, .) kink
within 1e-3, where the derivative is taken as 0.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_11719_gb300 import inputs as I  # noqa: E402
from tests.gpu_helpers import G_REL  # noqa: E402
from tests.test_gpu_repair import kinks  # noqa: E402


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_11719_gb300 import smppi
    return smppi


def _recovered_gradient(S, ctl, x0, V, go, box):
    """(V - V_out) / delta after one fixed step, and the mask of unclipped components."""
    delta = 0.02 / np.max(np.abs(go))
    Vout = torch.empty((1,) + V.shape, device="cuda")
    S.smppi_repair(ctl.h, 1, ctl.tensor(x0[None]), ctl.tensor(V[None]), Vout, 1, 0, delta)
    assert ctl.sync_status()[0] == S.OK
    Vo = Vout[0].cpu().numpy().astype(np.float64)
    Vd = V.astype(np.float64)
    lo, hi = box
    free = (np.abs(Vo - lo) > 1e-6) & (np.abs(Vo - hi) > 1e-6)
    return (Vd - Vo) / delta, free


def _compare(g, go, free):
    return np.linalg.norm((g - go)[free]) / max(np.linalg.norm(go[free]), 1e-12)


def test_block_gradient_cartesian(S, orc):
    sb = I.near_boundary_sequences(n_seq=48, T=100, seed=4)
    m = orc.Model(sb.params, sb.track)
    ctl = S.Controller(sb.params, sb.track, max_seq=1)
    box = (np.array(sb.params["u_min"]), np.array(sb.params["u_max"]))
    clean, worst = 0, 0.0
    for i in range(len(sb.x0)):
        Jo, go = orc.cost_grad(m, sb.x0[i], sb.V[i], 100, 0.0, 1.0)
        if Jo == 0.0 or kinks(orc, m, sb.x0[i], sb.V[i]):
            continue
        g, free = _recovered_gradient(S, ctl, sb.x0[i], sb.V[i], go, box)
        worst = max(worst, _compare(g, go, free))
        clean += 1
    ctl.close()
    print("block gradient (Cartesian), %d kink-free sequences: worst rel l2 %.2e" % (clean, worst))
    assert clean >= 8 and worst <= G_REL


def test_block_gradient_curvilinear(S, orc):
    sb = I.near_edge_curvilinear(32, 40, 9)
    m = orc.Model(sb.params, sb.track)
    ctl = S.Controller(sb.params, sb.track, max_seq=1)
    box = (np.array(sb.params["u_min"]), np.array(sb.params["u_max"]))
    a1 = 1 - float(np.float32(sb.params["alpha"]))
    w2 = float(np.float32(sb.params["half_width"])) ** 2
    clean, worst = 0, 0.0
    for i in range(len(sb.x0)):
        Jo, go = orc.cost_grad(m, sb.x0[i], sb.V[i], None, 0.0, 1.0)
        _, traj, _ = orc.rollout(m, sb.x0[i], sb.V[i], noisy=False)
        h = w2 - traj[:, 4] ** 2
        if Jo == 0.0 or np.any(np.abs(a1 * h[:-1] - h[1:]) < 1e-3):
            continue
        g, free = _recovered_gradient(S, ctl, sb.x0[i], sb.V[i], go, box)
        worst = max(worst, _compare(g, go, free))
        clean += 1
    ctl.close()
    print("block gradient (curvilinear), %d kink-free sequences: worst rel l2 %.2e"
          % (clean, worst))
    assert clean >= 6 and worst <= G_REL
