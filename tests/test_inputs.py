"""The seeded input generators: every workload's inputs are a function of the
seed alone (two calls give identical arrays, another seed other arrays), have
the shapes and dtypes the C ABI takes, and stay inside the ranges their
recipes state (control box, offsets from the centreline, track geometry)."""
import math

import numpy as np

from paper_2302_11719_gb300 import inputs as I


def test_single_problem_recipe():
    pr = I.single_problem(K=256, T=50)
    assert pr.track.shape == (I.N_TRACK, 2) and pr.track.dtype == np.float32
    assert pr.x0.dtype == np.float32 and pr.V.shape == (50, 2) and not pr.V.any()
    th = 2 * np.pi * np.arange(I.N_TRACK) / I.N_TRACK
    assert np.allclose(pr.track[:, 0], 20 * np.cos(th), atol=1e-5)
    assert np.allclose(pr.track[:, 1], 12 * np.sin(th), atol=1e-5)
    # counter-clockwise: positive signed area
    x, y = pr.track[:, 0].astype(np.float64), pr.track[:, 1].astype(np.float64)
    assert 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) > 0
    assert np.allclose(pr.x0, [5, 0, 0, 20, 0, math.pi / 2])


def test_near_boundary_sequences_seeded_and_in_range():
    a = I.near_boundary_sequences(256, 40, seed=3)
    b = I.near_boundary_sequences(256, 40, seed=3)
    c = I.near_boundary_sequences(256, 40, seed=4)
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.V, b.V)
    assert not np.array_equal(a.x0, c.x0)
    assert a.x0.shape == (256, 6) and a.V.shape == (256, 40, 2) and a.V.dtype == np.float32
    assert np.all(np.abs(a.V[..., 0]) <= 0.5) and np.all(np.abs(a.V[..., 1]) <= 1.0)
    assert np.all((a.x0[:, 0] >= 5) & (a.x0[:, 0] <= 8))
    # offsets from the ellipse: outside the inner half of the track, inside the edge
    X, Y = a.x0[:, 3].astype(np.float64), a.x0[:, 4].astype(np.float64)
    r = np.sqrt((X / 20) ** 2 + (Y / 12) ** 2)
    assert np.all(np.abs(r - 1) > 0.05)
    assert set(np.unique(a.side)) <= {-1.0, 1.0}


def test_near_edge_curvilinear_seeded_and_in_range():
    a = I.near_edge_curvilinear(64, 40, seed=7)
    b = I.near_edge_curvilinear(64, 40, seed=7)
    assert np.array_equal(a.x0, b.x0) and np.array_equal(a.V, b.V)
    assert a.params["state_kind"] == 1 and a.T == 40
    ey = a.x0[:, 4]
    assert np.all((np.abs(ey) >= 1.4) & (np.abs(ey) <= 1.8))
    assert np.array_equal(np.sign(ey), a.side.astype(np.float32))
    assert np.all(np.abs(a.V[..., 0]) <= 0.45) and np.all(np.abs(a.V[..., 1]) <= 0.9)


def test_uneven_instances_recipe():
    a = I.uneven_instances(64, seed=1)
    b = I.uneven_instances(64, seed=1)
    assert np.array_equal(a.K, b.K) and np.array_equal(a.tracks, b.tracks)
    assert np.all((a.K >= 64) & (a.K <= 16384)) and np.all((a.T >= 20) & (a.T <= 150))
    assert np.all((a.w >= 1.5) & (a.w <= 3.0))
    # no cusp on the inner boundary: the smallest radius of curvature exceeds 2 w
    assert np.all(np.minimum(a.a, a.b) ** 2 / np.maximum(a.a, a.b) > 2 * a.w)
    assert np.all([p["K"] == k and p["T"] == t for p, k, t in zip(a.params, a.K, a.T)])
