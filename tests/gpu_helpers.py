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
