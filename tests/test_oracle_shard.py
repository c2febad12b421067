"""Pins of the oracle's sharded update: Eq. 10-11 evaluated slice by slice over
a partition of the K rollouts and merged with the rescaling
c_g = exp(-(m_g - m)/lambda) (a log-sum-exp merge).

  * for partitions into 1, 2, 3 and 7 uneven contiguous slices the merged V+
    equals the oracle's single update over all K costs (a separate code path,
    pinned in test_oracle_update.py) to rounding;
  * the order of the slices does not matter;
  * shifting one slice's costs by a constant shifts its m_g and leaves eta_g
    and A_g unchanged (the min shift);
  * lambda -> 0: the merged update applies the noise of the global arg-min
    rollout, whichever slice holds it.
"""
import numpy as np

from paper_2302_11719_gb300 import inputs as I


def _setup(orc, K=96, T=12, lam=None):
    kw = {} if lam is None else {"lam": lam}
    pr = I.single_problem(K=K, T=T, **kw)
    m = orc.Model(pr.params, pr.track)
    rng = np.random.default_rng(9)
    V = rng.uniform(-0.2, 0.2, (T, 2))
    S, Vp = orc.mppi_step(m, pr.x0, V, 3, 5, nthreads=4)
    return m, V, S, Vp


def _cuts(K, n, rng):
    c = np.sort(rng.choice(np.arange(1, K), n - 1, replace=False))
    return np.concatenate([[0], c, [K]])


def test_merge_equals_single_update(orc):
    m, V, S, Vp = _setup(orc)
    rng = np.random.default_rng(2)
    for n in (1, 2, 3, 7):
        b = _cuts(m.K, n, rng)
        parts = [orc.partial(m, S[b[g]:b[g + 1]], b[g], 3, 5) for g in range(n)]
        Vm = orc.merge(m, parts, V)
        assert np.max(np.abs(Vm - Vp)) < 1e-13, n
        # the order of the slices does not matter
        Vr = orc.merge(m, parts[::-1], V)
        assert np.max(np.abs(Vr - Vp)) < 1e-13


def test_partial_min_shift(orc):
    m, V, S, _ = _setup(orc)
    a = orc.partial(m, S[10:40], 10, 3, 5)
    b = orc.partial(m, S[10:40] + 123.25, 10, 3, 5)
    assert b[0] == a[0] + 123.25
    # to rounding: S_k + c - (m + c) differs from S_k - m by an ulp of the costs (~1e3)
    assert np.max(np.abs(b[1:] - a[1:])) <= 1e-11 * np.max(np.abs(a[1:]))
    assert a[1] >= 1.0                     # the slice's arg-min has weight 1


def test_merge_small_lambda_selects_argmin(orc):
    m, V, S, _ = _setup(orc, lam=1e-6)
    k_star = int(np.argmin(S))
    b = [0, 30, 61, m.K]
    parts = [orc.partial(m, S[b[g]:b[g + 1]], b[g], 3, 5) for g in range(3)]
    Vm = orc.merge(m, parts, V)
    eps = orc.noise_block(m, 3, 5, [k_star])[0]
    lo, hi = np.array([-0.5, -1.0]), np.array([0.5, 1.0])
    assert np.allclose(Vm, np.clip(V + eps, lo, hi), atol=1e-12)
