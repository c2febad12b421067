"""Minimax fit of the polynomial behind the kernels' atan2 (device.cuh
atan2_poly, atan2_2 and atan2_2_lat).

After the octant reduction the kernels need atan(a) for a in [0, 1]; they
evaluate it as a p(a^2) with p of degree 8.  This script finds p by the Remez
exchange algorithm for the smallest maximum ABSOLUTE error of atan(a): with
s = a^2 it minimises max_s | sqrt(s) (p(s) - f(s)) | over s in [0, 1], where
f(s) = atan(sqrt(s)) / sqrt(s) (f(0) = 1), i.e. a weighted minimax fit with
weight sqrt(s).

    python atan_minimax.py      # prints the nine coefficients, highest first

The printed values, rounded to float32, are the ATAN_P0..8 constants of
device.cuh (the one copy); tests/test_atan_fit.py regenerates and compares them.
"""
from __future__ import annotations

import numpy as np

DEGREE = 8


def f(s):
    s = np.asarray(s, dtype=np.float64)
    out = np.empty_like(s)
    small = s < 1e-8
    r = np.sqrt(s[~small])
    out[~small] = np.arctan(r) / r
    ss = s[small]
    out[small] = 1.0 - ss / 3.0 + ss * ss / 5.0      # series of atan(a)/a in s = a^2
    return out


def weight(s):
    return np.sqrt(np.asarray(s, dtype=np.float64))


def poly(c, s):
    """c[0] + c[1] s + ... (ascending)."""
    return np.polynomial.polynomial.polyval(s, c)


def _solve(ref):
    """Coefficients c (ascending) and level E with w(x_i)(p(x_i) - f(x_i)) = (-1)^i E."""
    n = DEGREE + 1
    A = np.zeros((n + 1, n + 1))
    for i, x in enumerate(ref):
        A[i, :n] = weight(x) * x ** np.arange(n)
        A[i, n] = -((-1.0) ** i)
    b = weight(ref) * f(ref)
    sol = np.linalg.solve(A, b)
    return sol[:n], sol[n]


def _extrema(c, grid):
    """Alternating extrema of the weighted error on a dense grid, refined locally."""
    e = weight(grid) * (poly(c, grid) - f(grid))
    # local extrema of |e| including the end points
    idx = [0]
    for i in range(1, len(grid) - 1):
        if (e[i] - e[i - 1]) * (e[i + 1] - e[i]) <= 0 and e[i] != 0:
            idx.append(i)
    idx.append(len(grid) - 1)
    pts = []
    for i in idx:           # refine by a local golden-section search on |e|
        lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
        sgn = np.sign(e[i])
        for _ in range(60):
            m1, m2 = lo + (hi - lo) * 0.382, lo + (hi - lo) * 0.618
            g1 = sgn * weight(m1) * (poly(c, m1) - f(np.array([m1]))[0])
            g2 = sgn * weight(m2) * (poly(c, m2) - f(np.array([m2]))[0])
            if g1 > g2:
                hi = m2
            else:
                lo = m1
        x = 0.5 * (lo + hi) if 0 < i < len(grid) - 1 else grid[i]
        pts.append(x)
    pts = np.array(pts)
    ev = weight(pts) * (poly(c, pts) - f(pts))
    # keep one point per sign run (the largest |e| of the run)
    keep_x, keep_e = [], []
    for x, v in zip(pts, ev):
        if keep_e and np.sign(v) == np.sign(keep_e[-1]):
            if abs(v) > abs(keep_e[-1]):
                keep_x[-1], keep_e[-1] = x, v
        else:
            keep_x.append(x)
            keep_e.append(v)
    return np.array(keep_x), np.array(keep_e)


def fit(iterations: int = 40):
    """(coefficients ascending, max |weighted error|) of the minimax polynomial."""
    n = DEGREE + 2
    k = np.arange(n)
    # the weight vanishes at s = 0 (the error of atan there is 0 for every p), so
    # the reference points stay inside (0, 1]: Chebyshev points of the first kind
    ref = 0.5 - 0.5 * np.cos(np.pi * (k + 0.5) / n)
    ref[-1] = 1.0
    grid = np.linspace(0.0, 1.0, 20001)[1:]
    for _ in range(iterations):
        c, E = _solve(ref)
        xs, es = _extrema(c, grid)
        if len(xs) < n:
            break
        # choose n consecutive alternating extrema containing the largest one
        j = int(np.argmax(np.abs(es)))
        start = min(max(0, j - n // 2), len(xs) - n)
        new_ref = xs[start:start + n]
        if np.max(np.abs(new_ref - ref)) < 1e-15:
            break
        ref = new_ref
    c, E = _solve(ref)
    err = np.max(np.abs(weight(grid) * (poly(c, grid) - f(grid))))
    return c, err


def float32_coefficients():
    """The fit's coefficients rounded to float32, highest degree first (the
    Horner order of the kernels)."""
    c, _ = fit()
    return [float(np.float32(v)) for v in c[::-1]]


if __name__ == "__main__":
    c, err = fit()
    for v in c[::-1]:
        print("%.9e" % np.float32(v))
    print("max |atan(a) - a p(a^2)| on [0, 1]: %.3e" % err)
