"""Shared helpers of the GPU parity tests (tolerances and comparisons).

Tolerances (float32 CUDA path vs the float64 oracle):
  rollout costs S~ and states: 1e-4 relative (scale max(|oracle|, 1)), T <= 100;
  control update from identical costs: 1e-5 absolute;
  control update end to end: 1e-5 + 2 B_t, where B_t is the first-order effect
  of cost errors within their 1e-4 tolerance on the softmin average,
  B_t = sum_k w_k (1e-4 (|S_k| + 1) / lambda) |eps_kt - (V+_t - V_t)|, w = the
  oracle's normalised weights (all values from the oracle);
  repaired controls: 1e-4 absolute; gradients: 1e-3 relative l2.
"""
import numpy as np

S_REL = 1e-4
X_REL = 1e-4
V_UPD = 1e-5
V_REP = 1e-4
G_REL = 1e-3


def rel_err(gpu, ref, floor=1.0):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.max(np.abs(gpu - ref) / np.maximum(np.abs(ref), floor))


def update_bound(S, eps, omega_norm, Vplus, V, lam):
    """Per-(t, j) tolerance of the end-to-end V+ comparison (see module doc)."""
    dV = np.asarray(Vplus, np.float64) - np.asarray(V, np.float64)
    tau = S_REL * (np.abs(S) + 1.0) / lam                     # (K,)
    B = np.einsum("k,k,ktj->tj", omega_norm, tau, np.abs(eps - dV[None]))
    return V_UPD + 2.0 * B


def repair_compare(S, orc, params, track, x0s, Vs, n_iters, mode=1):
    """GPU smppi_repair against the oracle's repair (same mode) on each start:
    (flips, worst |V_safe - oracle| over the sequences without a flip).  A flip
    is a sequence whose iteration count differs or whose controls differ by
    more than V_REP: a line-search accept/reject decision that float32 and
    float64 take differently.  Asserts monotone GPU merits and P(V) at the
    start within S_REL."""
    import pytest
    import torch
    n = x0s.shape[0]
    ctl = S.Controller(params, track, max_seq=n)
    Vout = torch.empty((n, ctl.T, 2), device="cuda")
    mer = torch.empty((n, n_iters + 1), dtype=torch.float64, device="cuda")
    its = torch.empty(n, dtype=torch.int32, device="cuda")
    S.smppi_repair(ctl.h, n, ctl.tensor(x0s), ctl.tensor(Vs), Vout, n_iters, mode, 0.0, mer, its)
    st, bits = ctl.sync_status()
    assert st in (S.OK, S.ERR_STALLED), st
    Vout, mer, its = Vout.cpu().numpy(), mer.cpu().numpy(), its.cpu().numpy()
    m = orc.Model(params, track)
    flips, worst = 0, 0.0
    for i in range(n):
        Vo, mo, so, io = orc.repair(m, x0s[i], Vs[i], n_iters, mode=mode)
        assert np.all(np.diff(mer[i]) <= 1e-9 * (1 + mer[i][:-1]))     # monotone merit
        assert mer[i][0] == pytest.approx(mo[0], rel=S_REL, abs=1e-2)
        if io != its[i]:
            flips += 1
            continue
        e = np.max(np.abs(Vout[i] - Vo))
        if e > V_REP:
            flips += 1       # same iteration count but a different accepted trial step
            continue
        worst = max(worst, e)
    ctl.close()
    return flips, worst
