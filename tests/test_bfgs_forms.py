"""The two forms of the BFGS repair's inverse Hessian (reading c27): the dense
update H <- (I - rho s y') H (I - rho y s') + rho s s' applied pair by pair to
H0 = (s0'y0 / y0'y0) I, and the two-loop recursion over the stored pairs that
the GPU solver uses when the pairs fit its workspace slice, give the same
product H v (float64, random pairs with s'y > 0), also restricted to a set of
free coordinates (P_F H P_F g).  A plain-mathematics check of the identity the
stored-pair form rests on; the GPU forms are held to the oracle's BFGS by
tests/test_gpu_bfgs.py."""
import numpy as np


def _dense(S, Y, h0):
    n = S.shape[1]
    H = h0 * np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (y @ s)
        A = np.eye(n) - rho * np.outer(s, y)
        H = A @ H @ A.T + rho * np.outer(s, s)
    return H


def _two_loop(S, Y, h0, v):
    k = len(S)
    rho = [1.0 / (Y[i] @ S[i]) for i in range(k)]
    q = v.copy()
    alpha = np.zeros(k)
    for i in range(k - 1, -1, -1):
        alpha[i] = rho[i] * (S[i] @ q)
        q -= alpha[i] * Y[i]
    r = h0 * q
    for i in range(k):
        beta = rho[i] * (Y[i] @ r)
        r += (alpha[i] - beta) * S[i]
    return r


def _pairs(rng, n, k):
    S, Y = [], []
    M = rng.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)            # a positive definite curvature
    for _ in range(k):
        s = rng.normal(size=n)
        y = A @ s + 0.1 * rng.normal(size=n)
        if y @ s <= 0:
            y = -y
        S.append(s)
        Y.append(y)
    return np.array(S), np.array(Y)


def test_two_loop_equals_dense_update():
    rng = np.random.default_rng(0)
    for n, k in ((6, 1), (20, 4), (40, 11), (200, 19)):
        S, Y = _pairs(rng, n, k)
        h0 = (S[0] @ Y[0]) / (Y[0] @ Y[0])
        H = _dense(S, Y, h0)
        for _ in range(3):
            v = rng.normal(size=n)
            a, b = H @ v, _two_loop(S, Y, h0, v)
            assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(a)))


def test_two_loop_free_set_product():
    rng = np.random.default_rng(1)
    n, k = 30, 6
    S, Y = _pairs(rng, n, k)
    h0 = (S[0] @ Y[0]) / (Y[0] @ Y[0])
    H = _dense(S, Y, h0)
    g = rng.normal(size=n)
    free = rng.random(n) > 0.3
    want = np.where(free, H @ np.where(free, g, 0.0), 0.0)   # P_F H P_F g
    got = np.where(free, _two_loop(S, Y, h0, np.where(free, g, 0.0)), 0.0)
    assert np.max(np.abs(want - got)) <= 1e-10 * max(1.0, np.max(np.abs(want)))
