"""Pins of the oracle's BFGS repair (the solver Sec. IV-B names for Eq. 22;
variant: box projection, Armijo on the projected path, binding
coordinates held, restarts along the gradient step).

  * the inverse update H+ = (I - rho s y') H (I - rho y s') + rho s s' meets
    the secant equation H+ y = s, stays symmetric and keeps H positive definite
    when s'y > 0 (properties fixed by the definition, checked on random data);
    H+ - H has rank at most two and H+ v = H v for v orthogonal to s and H y;
  * the solver on quadratics 1/2 z'Az - b'z: the unconstrained minimiser
    A^-1 b inside a wide box (superlinear convergence to machine precision);
    the clipped minimiser for a diagonal A whose minimiser lies outside the
    box; the KKT conditions for a general A with active bounds;
  * on the repair objective: one BFGS iteration is exactly one projected
    gradient + Armijo iteration (mode 1), the merit never increases, and an
    already safe sequence (P = 0) is a fixed point with no iteration run.
"""
import numpy as np
import pytest

from paper_2302_11719_gb300 import inputs as I


def _spd(rng, n):
    M = rng.normal(size=(n, n))
    return M @ M.T + n * np.eye(n)


@pytest.mark.parametrize("n", [3, 8, 40])
def test_bfgs_update_secant_symmetry_pd(orc, n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        H = np.linalg.inv(_spd(rng, n))
        s = rng.normal(size=n)
        A = _spd(rng, n)
        y = A @ s                                   # s'y > 0 for an SPD A
        Hn = orc.bfgs_update(H, s, y)
        assert np.allclose(Hn @ y, s, rtol=1e-10, atol=1e-12 * np.abs(s).max())
        assert np.allclose(Hn, Hn.T, atol=1e-14 * np.abs(Hn).max())
        assert np.linalg.eigvalsh(0.5 * (Hn + Hn.T)).min() > 0.0


def test_bfgs_update_rank_two(orc):
    # For s'v = 0 the right factor leaves v alone, so H+ v = (I - rho s y') H v,
    # which is H v when also y'H v = (H y)'v = 0.
    rng = np.random.default_rng(7)
    n = 10
    H = np.linalg.inv(_spd(rng, n))
    s = rng.normal(size=n)
    y = _spd(rng, n) @ s
    Hn = orc.bfgs_update(H, s, y)
    assert np.linalg.matrix_rank(Hn - H, tol=1e-10 * np.abs(H).max()) <= 2
    # v orthogonal to s and to H y
    Q, _ = np.linalg.qr(np.stack([s, H @ y] + [rng.normal(size=n) for _ in range(n - 2)], 1))
    for k in range(2, n):
        v = Q[:, k]
        assert np.allclose(Hn @ v, H @ v, atol=1e-12)


@pytest.mark.parametrize("n", [6, 20])
def test_bfgs_quadratic_interior(orc, n):
    rng = np.random.default_rng(100 + n)
    A = _spd(rng, n)
    b = 5 * rng.normal(size=n)
    z_star = np.linalg.solve(A, b)
    lo, hi = np.full(n, -50.0), np.full(n, 50.0)
    assert np.all(np.abs(z_star) < 40)
    z, f, st, it = orc.bfgs_quadratic(A, b, lo, hi, np.ones(n), 100)
    assert np.max(np.abs(z - z_star)) <= 1e-9 * max(1.0, np.abs(z_star).max())
    assert np.all(np.diff(f[:it + 1]) <= 0.0)


@pytest.mark.parametrize("n", [6, 20, 40])
def test_bfgs_quadratic_clipped(orc, n):
    rng = np.random.default_rng(200 + n)
    d = rng.uniform(1.0, 5.0, n)
    b = 20 * rng.normal(size=n)
    lo, hi = -np.ones(n), np.ones(n)
    z, f, st, it = orc.bfgs_quadratic(np.diag(d), b, lo, hi, np.full(n, 0.3), 100)
    assert np.array_equal(z, np.clip(b / d, lo, hi)) or \
        np.max(np.abs(z - np.clip(b / d, lo, hi))) <= 1e-12


@pytest.mark.parametrize("n", [6, 20, 40])
def test_bfgs_quadratic_kkt(orc, n):
    rng = np.random.default_rng(300 + n)
    A = _spd(rng, n)
    b = 50 * rng.normal(size=n)
    lo, hi = -np.ones(n), np.ones(n)
    z, f, st, it = orc.bfgs_quadratic(A, b, lo, hi, np.full(n, 0.3), 200)
    g = A @ z - b
    assert np.all(z >= lo) and np.all(z <= hi)
    # KKT of the box problem: g_i = 0 on free coordinates, g_i >= 0 at the
    # lower bound, g_i <= 0 at the upper bound
    r = np.where(z <= lo, np.minimum(g, 0.0), np.where(z >= hi, np.maximum(g, 0.0), g))
    assert np.abs(r).max() <= 1e-6 * np.abs(b).max()
    assert ((z <= lo) | (z >= hi)).sum() >= 1          # the bounds are really active


@pytest.fixture(scope="module")
def seqs():
    return I.near_boundary_sequences(n_seq=24, T=40, seed=1)


@pytest.fixture(scope="module")
def model(orc, seqs):
    return orc.Model(seqs.params, seqs.track)


def test_bfgs_first_iteration_is_gradient_step(orc, seqs, model):
    for q in range(12):
        Va, ma, sa, ia = orc.repair(model, seqs.x0[q], seqs.V[q], 1, mode=1)
        Vb, mb, sb, ib = orc.repair(model, seqs.x0[q], seqs.V[q], 1, mode=2)
        assert np.array_equal(Va, Vb) and np.array_equal(ma, mb) and ia == ib and sa == sb


def test_bfgs_merit_monotone_and_reduces(orc, seqs, model):
    n_unsafe, n_safe_after = 0, 0
    for q in range(len(seqs.x0)):
        V2, m2, s2, i2 = orc.repair(model, seqs.x0[q], seqs.V[q], 10, mode=2)
        assert np.all(np.diff(m2) <= 0.0)
        assert m2[-1] == pytest.approx(orc.merit(model, seqs.x0[q], V2), rel=1e-12, abs=1e-12)
        assert np.all(V2[:, 0] >= -0.5) and np.all(V2[:, 0] <= 0.5)
        assert np.all(V2[:, 1] >= -1.0) and np.all(V2[:, 1] <= 1.0)
        if m2[0] > 0:
            n_unsafe += 1
            n_safe_after += m2[-1] == 0.0
    assert n_unsafe >= 10 and n_safe_after >= n_unsafe // 2


def test_bfgs_safe_sequence_is_fixed_point(orc, seqs, model):
    for q in range(len(seqs.x0)):
        if orc.merit(model, seqs.x0[q], seqs.V[q]) == 0.0:
            V2, m2, s2, i2 = orc.repair(model, seqs.x0[q], seqs.V[q], 5, mode=2)
            assert i2 == 0 and np.array_equal(V2, seqs.V[q].astype(np.float64)) and s2 == 0
            return
    pytest.skip("no safe sequence in the sample")
